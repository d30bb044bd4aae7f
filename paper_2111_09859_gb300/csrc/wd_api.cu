// wd_api.cu -- C ABI of libwd: grid creation (metrics, masks, line tables), the
// pseudo-time solver driver (Sec. 3.3) and the operator entry points.  Every step of the
// method runs in the kernels of wd_kernels.cu; this file only sequences launches, moves
// caller arrays in and out of the padded device layout and reads the convergence norms.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "wd_api_internal.h"
#include "wd_cart3d.h"
#include "wd_zfilter.h"
#include "wd_fused2d.h"
#include "wd_line2d.h"

using namespace wd;

namespace wd {
static thread_local std::string g_err;
wd_status set_error(wd_status s, const char* msg)
{
    g_err = msg;
    return s;
}
wd_status cuda_error(cudaError_t e, const char* where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return WD_ERR_CUDA;
}
}  // namespace wd

#define CK(...)                                                         \
    do {                                                                \
        cudaError_t _e = (__VA_ARGS__);                                 \
        if (_e != cudaSuccess) return wd::cuda_error(_e, #__VA_ARGS__); \
    } while (0)
#define ST(...)                                \
    do {                                       \
        wd_status _s = (__VA_ARGS__);          \
        if (_s != WD_OK) return _s;            \
    } while (0)

enum {
    W_PHIN, W_PHIS, W_ACC, W_DT, W_D0, W_D1, W_D2, W_U0, W_U1, W_U2, W_N0, W_N1, W_N2,
    W_LAP, W_KAP, W_LAD, W_T0, W_T1, W_ADV, W_NWORK
};

// the baseline upwind scheme takes its central terms (metrics, Laplacian, Poisson guess)
// from E2 (Sec. 3.2.1)
static inline int central_scheme(int s) { return s == WD_UW ? WD_E2 : s; }

struct wd_grid_s {
    Dims D;
    wd_grid_desc desc;
    cudaStream_t stream = nullptr;       // library-owned non-blocking stream (all work)
    cudaStream_t user_stream = nullptr;  // the caller's stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // stacked grids: extra streams for the parts of a batch that run side by side, and the
    // events that fork them from and join them to `stream`
    static const int NPART = 4;
    cudaStream_t pst[NPART - 1] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[NPART - 1] = {};
    int es = 8;                 // bytes per state element
    size_t bytes = 0;
    double* xyz = nullptr;      // 3 padded coordinate arrays
    double* xi_d = nullptr;     // 9 padded arrays
    double* J_d = nullptr;
    double* dx_d = nullptr;     // 3 padded arrays
    void* xi_m = nullptr;       // metrics in the metric precision (aliases xi_d for double)
    int xi_alias = 1;
    void* sig1 = nullptr;
    void* sig2 = nullptr;
    void* lads = nullptr;       // 3 arrays
    double lads_exp = -1.0;
    double* ffr = nullptr;      // 6 x fmax spacing ratios
    long long fmax = 0;
    uint8_t* wall = nullptr;
    uint8_t* mask = nullptr;
    void* dval = nullptr;
    long long nactive = 0;
    int batch = 1;                       // stacked 2-D grids (n[2] in 2-D)
    std::vector<long long> nact;         // active nodes per stacked grid
    void* w[W_NWORK] = {};
    double* partial = nullptr;
    void* ztab = nullptr;       // Thomas factors of the filter along direction 2 (3 N values)
    double ztab_key = -1.0;     // alpha_f they were built for
    unsigned* counter = nullptr;
    double* result = nullptr;
    double* hres = nullptr;     // pinned
    unsigned long long* dcount = nullptr;
    int nred = 0;
    int npartial = 0;           // capacity of `partial` in blocks
    int force_generic = 0;      // WD_FORCE_GENERIC=1 at creation: never use the fused path
    int part_off = 0;           // WD_PART_OFF=1 at creation: fused 2-D path with PCR passes
    int line_off = 0;           // WD_LINE2D_OFF=1 at creation: fused 2-D path without the
                                // line-resident passes (per-operator partition passes)
    int tuned = 0;              // autotuner ran for this grid
    int tune_stage_threads = 0; // chosen block size of the 2-D stage kernel (0: default)
    int tune_by = 0;            // chosen block rows of the Cartesian stencil kernels (0: default)
    int tune_zf = 1;            // direction-2 filter + commit of 3-D grids: 1 streamed, 0 partition pass
    int tune_parts = 0;         // chosen number of parts of a stacked batch (line-resident path)
    int cart = 0;               // uniform Cartesian 3-D grid (diagonal constant metrics)
    double h[3] = {0, 0, 0};    // its spacings
    HostLineTab dtab[3], ftab[3], etab[3];
    // CUDA graphs of n pseudo steps, one per kind (HJ, Poisson), reused while the launch
    // arguments they captured are unchanged: same n, same parameters, same table generation
    unsigned gen = 0;                    // bumped when tables, scales or geometry change
    cudaGraphExec_t gx[2] = {nullptr, nullptr};
    int gx_n[2] = {0, 0};
    unsigned gx_gen[2] = {0, 0};
    wd_solve_params gx_p[2];
    // CUDA graph of two level-set steps, reused while F, dt and the geometry are unchanged
    cudaGraphExec_t lsx = nullptr;
    double ls_F = 0.0, ls_dt = 0.0;
    unsigned ls_gen = 0;
    // kernel timer (wd_profile)
    int prof_on = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_used;   // (class, index of the start event; stop = +1)
    double prof_ms[WD_K_NCLASS] = {};
    long long prof_n[WD_K_NCLASS] = {};
};

static cudaError_t prof_flush(wd_grid g)
{
    if (g->ev_used.empty()) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return e;
    for (auto& u : g->ev_used) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, g->ev_pool[u.second], g->ev_pool[u.second + 1]);
        if (e != cudaSuccess) return e;
        g->prof_ms[u.first] += ms;
        g->prof_n[u.first] += 1;
    }
    g->ev_used.clear();
    return cudaSuccess;
}

// brackets one launch with events when the timer is on
struct ProfScope {
    wd_grid g;
    int cls, idx = -1;
    ProfScope(wd_grid g_, int c) : g(g_), cls(c)
    {
        if (!g->prof_on) return;
        if (2 * (g->ev_used.size() + 1) > g->ev_pool.size()) {
            if (g->ev_pool.size() < 8192) {
                size_t old = g->ev_pool.size();
                g->ev_pool.resize(old + 512);
                for (size_t i = old; i < g->ev_pool.size(); i++) cudaEventCreate(&g->ev_pool[i]);
            } else if (prof_flush(g) != cudaSuccess) {
                return;
            }
        }
        idx = (int)(2 * g->ev_used.size());
        cudaEventRecord(g->ev_pool[idx], g->stream);
    }
    ~ProfScope()
    {
        if (idx < 0) return;
        cudaEventRecord(g->ev_pool[idx + 1], g->stream);
        g->ev_used.push_back({cls, idx});
    }
};

// metric type of the pseudo-step loop: FP64 only for the FP64 state.  FP32_METRIC64 computes
// the metric Jacobians in FP64 (create time) and runs the loop in FP32 on their rounded
// values; FP32 also takes the coordinate derivatives of the metrics in FP32
static bool metric_double(int prec) { return prec == WD_FP64; }

// Every call runs on the grid's own stream (graph capture needs a non-legacy stream), ordered
// after the work already queued on the caller's stream; on exit the caller's stream waits
// for the call's work, so the caller sees stream-ordered semantics on its own stream.
struct StreamGuard {
    wd_grid g;
    explicit StreamGuard(wd_grid g_) : g(g_)
    {
        cudaEventRecord(g->ev_in, g->user_stream);
        cudaStreamWaitEvent(g->stream, g->ev_in, 0);
    }
    ~StreamGuard()
    {
        cudaEventRecord(g->ev_out, g->stream);
        cudaStreamWaitEvent(g->user_stream, g->ev_out, 0);
    }
};

static size_t footprint_bytes(const wd_grid_desc* d)
{
    long long pitch = (d->n[0] + 31) / 32 * 32;
    long long total = pitch * d->n[1] * d->n[2];
    size_t es = d->precision == WD_FP64 ? 8 : 4;
    size_t ms = metric_double(d->precision) ? 8 : 4;
    size_t b = 0;
    b += (size_t)total * 8 * (3 + 9 + 1 + 3);          // xyz, xi_d, J, dx
    if (!metric_double(d->precision)) b += (size_t)total * 4 * 9;
    b += (size_t)total * ms * (2 + 3);                  // sig1, sig2, lads
    b += (size_t)total * (2 + es);                      // wall, mask, dval
    b += (size_t)total * es * (W_NWORK - (d->scheme == WD_UW ? 0 : 1));   // W_ADV: baseline only
    long long fmax = 0;
    for (int k = 0; k < 3; k++) {
        long long f = (long long)d->n[(k + 1) % 3] * d->n[(k + 2) % 3];
        if (f > fmax) fmax = f;
    }
    b += (size_t)fmax * 6 * 8;
    for (int k = 0; k < d->ndim; k++) {
        int L = 0;
        while ((1 << L) < d->n[k]) L++;
        b += 3 * (size_t)(2 * L + 3) * d->n[k] * 12;
    }
    return b;
}

static wd_status validate_desc(const wd_grid_desc* d)
{
    if (!d) return set_error(WD_ERR_INVALID_ARG, "desc is NULL");
    if (d->ndim != 2 && d->ndim != 3) return set_error(WD_ERR_INVALID_ARG, "ndim must be 2 or 3");
    if (d->n[2] < 1) return set_error(WD_ERR_INVALID_ARG, "n[2] must be >= 1 (grids stacked in 2-D)");
    if (d->ndim == 2 && d->n[2] > 1) {
        auto ok = [](int k) { return k == WD_BC_PERIODIC || k == WD_BC_WALL; };
        if (!ok(d->bc_lo[0]) || !ok(d->bc_hi[0]))
            return set_error(WD_ERR_INVALID_ARG,
                             "stacked 2-D grids need periodic or wall faces in direction 0");
    }
    for (int k = 0; k < d->ndim; k++) {
        if (d->n[k] < 8) return set_error(WD_ERR_INVALID_ARG, "every direction needs >= 8 nodes");
        if (d->n[k] > 2048) return set_error(WD_ERR_INVALID_ARG, "at most 2048 nodes per direction");
        int lo = d->bc_lo[k], hi = d->bc_hi[k];
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3)
            return set_error(WD_ERR_INVALID_ARG, "unknown boundary kind");
        if ((lo == WD_BC_PERIODIC) != (hi == WD_BC_PERIODIC))
            return set_error(WD_ERR_INVALID_ARG, "periodic must be set on both faces");
    }
    if (d->precision < 0 || d->precision > 2) return set_error(WD_ERR_INVALID_ARG, "bad precision");
    if (d->scheme < WD_E2 || d->scheme > WD_UW) return set_error(WD_ERR_INVALID_ARG, "bad scheme");
    if (d->scheme == WD_UW && d->ndim == 2 && d->n[2] > 1)
        return set_error(WD_ERR_INVALID_ARG, "the upwind baseline runs on single grids (the generic path)");
    if (!(d->L_ref > 0.0)) return set_error(WD_ERR_INVALID_ARG, "L_ref must be positive");
    long long tot = (long long)((d->n[0] + 31) / 32 * 32) * d->n[1] * d->n[2];
    if (tot > (1LL << 31)) return set_error(WD_ERR_INVALID_ARG, "grid too large");
    return WD_OK;
}

static wd_status dmalloc(wd_grid g, void** p, size_t bytes)
{
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(WD_ERR_OOM, "cudaMalloc failed");
    }
    g->bytes += bytes;
    return WD_OK;
}

// dense caller array <-> padded device array (either side may be host or device memory)
static cudaError_t to_padded(wd_grid g, void* dst, const void* src, size_t es)
{
    const Dims& D = g->D;
    return cudaMemcpy2DAsync(dst, (size_t)D.pitch * es, src, (size_t)D.n[0] * es, (size_t)D.n[0] * es,
                             (size_t)D.n[1] * D.n[2], cudaMemcpyDefault, g->stream);
}
static cudaError_t from_padded(wd_grid g, void* dst, const void* src, size_t es)
{
    const Dims& D = g->D;
    return cudaMemcpy2DAsync(dst, (size_t)D.n[0] * es, src, (size_t)D.pitch * es, (size_t)D.n[0] * es,
                             (size_t)D.n[1] * D.n[2], cudaMemcpyDefault, g->stream);
}

static void release(wd_grid g)
{
    if (!g) return;
    cudaFree(g->xyz);
    cudaFree(g->xi_d);
    cudaFree(g->J_d);
    cudaFree(g->dx_d);
    if (!g->xi_alias) cudaFree(g->xi_m);
    cudaFree(g->sig1);
    cudaFree(g->sig2);
    cudaFree(g->lads);
    cudaFree(g->ffr);
    cudaFree(g->wall);
    cudaFree(g->mask);
    cudaFree(g->dval);
    for (int k = 0; k < W_NWORK; k++) cudaFree(g->w[k]);
    cudaFree(g->partial);
    cudaFree(g->counter);
    cudaFree(g->result);
    cudaFree(g->ztab);
    cudaFree(g->dcount);
    if (g->hres) cudaFreeHost(g->hres);
    for (int k = 0; k < 3; k++) {
        free_line_table(g->dtab[k]);
        free_line_table(g->ftab[k]);
        free_line_table(g->etab[k]);
    }
    for (auto& e : g->ev_pool) cudaEventDestroy(e);
    for (int k = 0; k < 2; k++)
        if (g->gx[k]) cudaGraphExecDestroy(g->gx[k]);
    if (g->lsx) cudaGraphExecDestroy(g->lsx);
    if (g->ev_in) cudaEventDestroy(g->ev_in);
    if (g->ev_out) cudaEventDestroy(g->ev_out);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    for (int k = 0; k < wd_grid_s::NPART - 1; k++) {
        if (g->ev_join[k]) cudaEventDestroy(g->ev_join[k]);
        if (g->pst[k]) cudaStreamDestroy(g->pst[k]);
    }
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

// ------------------------------------------------------------------------------------
// autotuner: the launch shapes that do not change results (block size of the pointwise
// stage kernel, block rows of the Cartesian stencil kernels) are timed on the grid's own
// arrays before its first pseudo step and cached per grid shape for the process, so pooled
// and served grids of a known shape start tuned.  WD_AUTOTUNE=0 keeps the defaults.
// ------------------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;

static bool autotune_enabled()
{
    const char* e = std::getenv("WD_AUTOTUNE");
    return !(e && e[0] == '0');
}

// average device time of one call of fn on stream st (one untimed call first, then three)
template <typename F>
static float time_calls(cudaStream_t st, F&& fn)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return INFINITY;
    }
    fn();
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; r++) fn();
    cudaEventRecord(e1, st);
    float ms = INFINITY;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaGetLastError();
        ms = INFINITY;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / 3.0f;
}

// the cached choice for key, else the fastest candidate (timed by time_of) stored under key
template <typename F>
static int tune_choice(const std::string& key, std::initializer_list<int> cand, F&& time_of)
{
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return it->second;
    }
    int best = *cand.begin();
    float tb = INFINITY;
    for (int c : cand) {
        const float t = time_of(c);
        if (t < tb) {
            tb = t;
            best = c;
        }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    return best;
}

// ------------------------------------------------------------------------------------
// solver, templated on state precision T and metric precision M
// ------------------------------------------------------------------------------------

template <typename T, typename M>
struct Solver {
    wd_grid g;
    const wd_solve_params* p;
    cudaStream_t st;
    const Dims& D;
    Solver(wd_grid g_, const wd_solve_params* p_) : g(g_), p(p_), st(g_->stream), D(g_->D) {}

    T* W(int k) { return (T*)g->w[k]; }
    const M* xi() { return (const M*)g->xi_m; }

    wd_status ensure_filter(double al)
    {
        for (int d = 0; d < D.ndim; d++) {
            HostLineTab& t = g->ftab[d];
            if (t.valid && t.key == al) continue;
            std::vector<double> a, c;
            int imp;
            filter_rows(al, D.n[d], D.per[d], a, c, imp);
            ST(build_line_table(D.n[d], D.per[d], a, c, imp, t));
            t.key = al;
            g->gen++;
        }
        if (D.ndim == 3 && !D.per[2] && g->ztab_key != al) {
            // the streamed direction-2 pass: the filter rows' Thomas factors in the state precision
            const int N = D.n[2];
            std::vector<double> f(3 * (size_t)N);
            zfilter_factors(al, N, f.data());
            std::vector<T> ft(f.begin(), f.end());
            if (!g->ztab) CK(cudaMalloc(&g->ztab, 3 * (size_t)N * sizeof(double)));
            CK(cudaMemcpy(g->ztab, ft.data(), ft.size() * sizeof(T), cudaMemcpyHostToDevice));
            g->ztab_key = al;
            g->gen++;
        }
        return WD_OK;
    }
    wd_status ensure_lads(double ex)
    {
        if (g->lads_exp == ex) return WD_OK;
        CK(launch_lad_scale<M>(D, g->xi_d, g->dx_d, ex, (M*)g->lads, st));
        g->lads_exp = ex;
        g->gen++;
        return WD_OK;
    }

    LineOp op_deriv() const
    {
        LineOp op;
        std::memset(&op, 0, sizeof(op));
        op.kind = OPK_DERIV;
        op.scheme = central_scheme(g->desc.scheme);
        return op;
    }
    static wd_status op_filter(double al, LineOp& op)
    {
        std::memset(&op, 0, sizeof(op));
        op.kind = OPK_FILTER;
        for (int hw = 1; hw <= 5; hw++)
            if (!filter_coefficients(hw, al, op.fa[hw]))
                return set_error(WD_ERR_INVALID_ARG, "filter coefficients");
        op.fa[0][0] = 1.0;
        op.fa[0][1] = al;     // alpha_f, used by the delta-form right-hand side
        return WD_OK;
    }

    wd_status deriv_dir(int d, const T* in, T* out)
    {
        Fields<T> f;
        std::memset(&f, 0, sizeof(f));
        f.in[0] = in;
        f.out[0] = out;
        ProfScope ps(g, WD_K_DERIV);
        CK(launch_line<T, M>(D, d, g->dtab[d], op_deriv(), 1, 0, f, nullptr, 0, 0, st));
        return WD_OK;
    }
    wd_status filter_dir(int d, double al, const T* in, T* out)
    {
        ST(ensure_filter(al));
        LineOp op;
        ST(op_filter(al, op));
        Fields<T> f;
        std::memset(&f, 0, sizeof(f));
        f.in[0] = in;
        f.out[0] = out;
        ProfScope ps(g, WD_K_FILTER);
        CK(launch_line<T, M>(D, d, g->ftab[d], op, 1, 0, f, nullptr, 0, 0, st));
        return WD_OK;
    }

    // D_l phi for every l, then U (and n); Laplacian (and curvature) as metric-weighted
    // divergences of U (and n), Eq. 9 / Eq. 25
    wd_status grad_parts(const T* phi, bool curv)
    {
        for (int l = 0; l < D.ndim; l++) ST(deriv_dir(l, phi, W(W_D0 + l)));
        T* Dl[3] = {W(W_D0), W(W_D1), W(W_D2)};
        T* U[3] = {W(W_U0), W(W_U1), W(W_U2)};
        T* nv[3] = {W(W_N0), W(W_N1), W(W_N2)};
        ProfScope ps(g, WD_K_POINT);
        CK(launch_grad<T, M>(D, Dl, xi(), U, curv ? nv : nullptr, p ? p->eps0 : 1e-8, st));
        return WD_OK;
    }
    wd_status div_parts(bool curv)
    {
        int nd = D.ndim;
        for (int l = 0; l < nd; l++) {
            Fields<T> f;
            std::memset(&f, 0, sizeof(f));
            for (int m = 0; m < nd; m++) {
                f.in[m] = W(W_U0 + m);
                if (curv) f.in[nd + m] = W(W_N0 + m);
            }
            f.out[0] = W(W_LAP);
            f.out[1] = W(W_KAP);
            ProfScope ps(g, WD_K_DIV);
            CK(launch_line<T, M>(D, l, g->dtab[l], op_deriv(), curv ? 2 * nd : nd, 1, f, xi(), nd,
                                 l > 0, st));
        }
        return WD_OK;
    }
    // smoothed C |sum_l s_l d4_l(phi)| (Eq. 7); returns the buffer holding it
    wd_status lad_part(const T* phi, T** out)
    {
        ST(ensure_lads(p->lad_exp));
        {
            ProfScope ps(g, WD_K_POINT);
            CK(launch_lad_raw<T, M>(D, phi, (const M*)g->lads, p->C_lad, W(W_T0), st));
        }
        LineOp op;
        std::memset(&op, 0, sizeof(op));
        op.kind = OPK_GAUSS;
        T* a = W(W_T0);
        T* b = W(W_T1);
        for (int l = 0; l < D.ndim; l++) {
            Fields<T> f;
            std::memset(&f, 0, sizeof(f));
            f.in[0] = a;
            f.out[0] = b;
            ProfScope ps(g, WD_K_GAUSS);
            CK(launch_line<T, M>(D, l, g->etab[l], op, 1, 0, f, nullptr, 0, 0, st));
            T* t = a;
            a = b;
            b = t;
        }
        *out = a;
        return WD_OK;
    }

    wd_status bc(T* phi, bool poisson)
    {
        for (int d = 0; d < D.ndim; d++) {
            int lo = g->desc.bc_lo[d], hi = g->desc.bc_hi[d];
            bool any = (lo == WD_BC_FARFIELD || lo == WD_BC_NEUMANN || hi == WD_BC_FARFIELD ||
                        hi == WD_BC_NEUMANN);
            if (!any) continue;
            if (poisson) {
                if (lo == WD_BC_FARFIELD) lo = WD_BC_NEUMANN;
                if (hi == WD_BC_FARFIELD) hi = WD_BC_NEUMANN;
            }
            ProfScope ps(g, WD_K_BC);
            CK(launch_bc_face<T>(D, d, lo, hi, g->ffr + (2 * d) * g->fmax, g->ffr + (2 * d + 1) * g->fmax,
                                 phi, st));
        }
        ProfScope ps(g, WD_K_BC);
        CK(launch_bc_mask<T>(D, g->mask, poisson ? nullptr : (const T*)g->dval, phi, st));
        return WD_OK;
    }

    // the boundary conditions of bc() for a single 2-D grid whose interior Dirichlet nodes are
    // already reset (after a Cartesian stage): one launch
    wd_status bc_faces2d(T* phi, bool poisson)
    {
        int klo[2], khi[2];
        const double *rlo[2], *rhi[2];
        for (int d = 0; d < 2; d++) {
            klo[d] = g->desc.bc_lo[d];
            khi[d] = g->desc.bc_hi[d];
            if (poisson) {
                if (klo[d] == WD_BC_FARFIELD) klo[d] = WD_BC_NEUMANN;
                if (khi[d] == WD_BC_FARFIELD) khi[d] = WD_BC_NEUMANN;
            }
            rlo[d] = g->ffr + (2 * d) * g->fmax;
            rhi[d] = g->ffr + (2 * d + 1) * g->fmax;
        }
        ProfScope ps(g, WD_K_BC);
        CK(launch_bc_faces2d<T>(D, klo, khi, rlo, rhi, g->mask, (const T*)g->dval, poisson, phi, st));
        return WD_OK;
    }

    StageArgs<T, M> stage_args(const T* src, T* dst, bool poisson, const T* lad)
    {
        StageArgs<T, M> a;
        a.src = src;
        a.dst = dst;
        a.phin = W(W_PHIN);
        a.acc = W(W_ACC);
        a.dt = W(W_DT);
        a.U[0] = W(W_U0);
        a.U[1] = W(W_U1);
        a.U[2] = W(W_U2);
        a.lap = W(W_LAP);
        a.kap = W(W_KAP);
        a.lad = lad;
        a.adv = nullptr;
        a.sig1 = (const M*)g->sig1;
        a.sig2 = (const M*)g->sig2;
        a.eps = p->eps;
        a.cfl = p->cfl;
        a.equation = p->equation;
        a.curvature = p->curvature;
        a.poisson = poisson;
        return a;
    }

    wd_status rhs_into(const T* src, T* dst, bool poisson, int stage)
    {
        bool curv = !poisson && p->curvature;
        ST(grad_parts(src, curv));
        ST(div_parts(curv));
        T* lad = nullptr;
        if (!poisson && p->equation == WD_HJ_LAD) ST(lad_part(src, &lad));
        StageArgs<T, M> a = stage_args(src, dst, poisson, lad);
        ProfScope ps(g, WD_K_POINT);
        if (!poisson && g->desc.scheme == WD_UW) {
            CK(launch_uw_adv<T, M>(D, src, xi(), uw_cart(), W(W_ADV), st));
            a.adv = W(W_ADV);
        }
        CK(launch_stage<T, M>(D, a, stage, st));
        return WD_OK;
    }

    // fused 2-D path: direction-0 faces periodic or walls (all far-field handling happens
    // along direction-1 lines), see wd_fused2d.cu
    bool fused2d() const
    {
        if (D.ndim != 2 || g->force_generic || g->desc.scheme == WD_UW) return false;
        auto ok = [](int k) { return k == WD_BC_PERIODIC || k == WD_BC_WALL; };
        return ok(g->desc.bc_lo[0]) && ok(g->desc.bc_hi[0]);
    }

    F2Args<T, M> f2_args(bool poisson)
    {
        F2Args<T, M> a;
        std::memset(&a, 0, sizeof(a));
        a.D = D;
        a.scheme = g->desc.scheme;
        a.dtab0 = g->dtab[0].template view<T>();
        a.dtab1 = g->dtab[1].template view<T>();
        if (p->filter) a.ftab1 = g->ftab[1].template view<T>();
        a.xi = xi();
        a.lads = (const M*)g->lads;
        a.sig1 = (const M*)g->sig1;
        a.sig2 = (const M*)g->sig2;
        a.phin = W(W_PHIN);
        a.phin_w = W(W_PHIN);
        a.acc = W(W_ACC);
        a.dtv = W(W_DT);
        a.D0 = W(W_D0);
        a.D1 = W(W_D1);
        a.L0 = W(W_N0);
        a.L1 = W(W_N1);
        a.LAP0 = W(W_LAP);
        a.LAP1 = W(W_U0);
        a.KAP0 = W(W_KAP);
        a.KAP1 = W(W_U1);
        a.G0 = W(W_LAD);
        a.mask = g->mask;
        a.dval = (const T*)g->dval;
        a.ffr_lo = g->ffr + 2 * g->fmax;
        a.ffr_hi = g->ffr + 3 * g->fmax;
        a.bclo1 = g->desc.bc_lo[1];
        a.bchi1 = g->desc.bc_hi[1];
        a.eps = p->eps;
        a.cfl = p->cfl;
        a.C_lad = p->C_lad;
        a.eps0 = p->eps0;
        a.alpha_f = p->alpha_f;
        a.equation = p->equation;
        a.curvature = p->curvature;
        a.lad = p->equation == WD_HJ_LAD && !poisson;
        a.poisson = poisson;
        a.filter = p->filter;
        a.partial = g->partial;
        a.counter = g->counter;
        a.result = g->result;
        a.max_partials = g->npartial;
        a.batch = g->batch;
        a.stage_threads = g->tune_stage_threads;
        return a;
    }

    // the warp partition passes apply when every line length of the grid has tables
    bool part2d(const F2Args<T, M>& a) const
    {
        if (g->force_generic || g->part_off) return false;
        for (int d = 0; d < 2; d++) {
            const PartTab<T> dt = g->dtab[d].template pview<T>();
            if (!p2_supported(a, dt, F2_DERIV, d) || !p2_supported(a, dt, F2_DIV, d)) return false;
            if (p->filter) {
                const PartTab<T> ft = g->ftab[d].template pview<T>();
                if (!p2_supported(a, ft, d == 0 ? P2_FILTER0 : F2_FILTER, d)) return false;
            }
        }
        return true;
    }

    // the line-resident passes (wd_line2d.cuh) apply to the central schemes up to half width 2
    // when both line lengths have partition tables and the filter passes do too
    bool line2d(const F2Args<T, M>& a, bool poisson) const
    {
        if (g->line_off || !part2d(a)) return false;
        const int sch = g->desc.scheme;
        if (sch != WD_E2 && sch != WD_E4 && sch != WD_C4 && sch != WD_C6) return false;
        const int nf = p->curvature && !poisson ? 4 : 2;
        return l2_supported<T, M>(D, g->dtab[0].template pview<T>(), g->dtab[1].template pview<T>(), nf);
    }

    L2Args<T, M> l2_args(bool poisson)
    {
        L2Args<T, M> a;
        std::memset(&a, 0, sizeof(a));
        a.D = D;
        switch (g->desc.scheme) {   // interior rows of Eq. 16: a1 (f+1 - f-1) + a2 (f+2 - f-2)
        case WD_E2: a.a1 = T(0.5); a.a2 = T(0); break;
        case WD_E4: a.a1 = T(2.0 / 3.0); a.a2 = T(-1.0 / 12.0); break;
        case WD_C4: a.a1 = T(0.75); a.a2 = T(0); break;
        default: a.a1 = T(7.0 / 9.0); a.a2 = T(1.0 / 36.0); break;   // C6
        }
        a.implicit = g->dtab[0].implicit;
        a.xi = xi();
        a.lads = (const M*)g->lads;
        a.sig1 = (const M*)g->sig1;
        a.sig2 = (const M*)g->sig2;
        a.phin = W(W_PHIN);
        a.acc = W(W_ACC);
        a.dtv = W(W_DT);
        a.D0 = W(W_D0);
        a.D1 = W(W_D1);
        a.L1 = W(W_N1);
        a.LAP0 = W(W_LAP);
        a.KAP0 = W(W_KAP);
        a.G0 = W(W_LAD);
        a.mask = g->mask;
        a.dval = (const T*)g->dval;
        a.ffr_lo = g->ffr + 2 * g->fmax;
        a.ffr_hi = g->ffr + 3 * g->fmax;
        a.bclo1 = g->desc.bc_lo[1];
        a.bchi1 = g->desc.bc_hi[1];
        a.eps = p->eps;
        a.cfl = p->cfl;
        a.C_lad = p->C_lad;
        a.eps0 = p->eps0;
        a.equation = p->equation;
        a.lad = p->equation == WD_HJ_LAD && !poisson;
        a.poisson = poisson;
        a.filter = p->filter;
        if (p->filter) {
            LineOp op;
            if (op_filter(p->alpha_f, op) != WD_OK) a.filter = 0;
            for (int hw = 1; hw <= 5; hw++)
                for (int m = 1; m <= hw; m++) a.cf[hw][m] = T(0.5 * op.fa[hw][m] - (m == 1 ? p->alpha_f : 0.0));
        }
        a.phin_w = W(W_PHIN);
        a.commit = 1;
        a.fdir = 1;
        a.partial = g->partial;
        a.counter = g->counter;
        a.result = g->result;
        a.max_partials = g->npartial;
        a.batch = g->batch;
        return a;
    }

    // Y0, four (X, Y) stage pairs, the direction-0 filter (FX), the direction-1 filter with the
    // BCs, change norms and commit (FY): 10 launches.  A stacked batch may run as `parts`
    // contiguous ranges of its grids, each on its own stream (forked from and joined to the
    // grid's stream, so a CUDA graph capture records them as parallel branches): the grids are
    // independent, and the launches of one part fill the partly empty last wave of another's.
    // Every node and every per-grid norm is computed identically for any number of parts.
    wd_status line2d_seq(L2Args<T, M> a, bool poisson, cudaStream_t s0)
    {
        const PartTab<T> t0 = g->dtab[0].template pview<T>(), t1 = g->dtab[1].template pview<T>();
        const int nf = p->curvature && !poisson ? 4 : 2;
        a.src = W(W_PHIN);
        {
            ProfScope ps(g, WD_K_DERIV);
            CK(l2_launch<T, M>(a, t1, L2_Y0, nf, s0));
        }
        for (int s = 0; s < 4; s++) {
            a.src = stage_src(s);
            a.dst = stage_dst(s);
            a.stage = s;
            a.next = s < 3;
            {
                ProfScope ps(g, WD_K_LINE0);
                CK(l2_launch<T, M>(a, t0, L2_X, nf, s0));
            }
            {
                ProfScope ps(g, WD_K_LINE1);
                CK(l2_launch<T, M>(a, t1, L2_Y, nf, s0));
            }
        }
        a.src = stage_dst(3);
        a.dst = stage_dst(3);
        if (p->filter) {
            ProfScope ps(g, WD_K_FILTER);
            CK(l2_launch<T, M>(a, g->ftab[0].template pview<T>(), L2_FX, nf, s0));
        }
        ProfScope ps(g, WD_K_NORM);
        CK(l2_launch<T, M>(a, p->filter ? g->ftab[1].template pview<T>() : t1, L2_FY, nf, s0));
        return WD_OK;
    }

    // parts of a stacked batch: WD_BATCH_PARTS (1..4) when set, else the autotuner's choice;
    // one under the kernel timer, which times the grid's own stream only
    int line2d_parts() const
    {
        if (g->prof_on || g->batch < 2 || !g->ev_fork) return 1;
        int n = g->tune_parts > 0 ? g->tune_parts : 1;
        if (const char* e = std::getenv("WD_BATCH_PARTS")) n = std::atoi(e);
        return std::max(1, std::min(n, std::min(g->batch, (int)wd_grid_s::NPART)));
    }

    wd_status step_line2d(bool poisson, int parts)
    {
        L2Args<T, M> a = l2_args(poisson);
        if (parts <= 1) {
            a.kbeg = 0;
            a.kcnt = g->batch;
            a.counter = g->counter;
            return line2d_seq(a, poisson, st);
        }
        CK(cudaEventRecord(g->ev_fork, st));
        for (int k = 1; k < parts; k++) CK(cudaStreamWaitEvent(g->pst[k - 1], g->ev_fork, 0));
        for (int k = 0; k < parts; k++) {
            a.kbeg = k * g->batch / parts;
            a.kcnt = (k + 1) * g->batch / parts - a.kbeg;
            a.counter = g->counter + k;
            ST(line2d_seq(a, poisson, k == 0 ? st : g->pst[k - 1]));
        }
        for (int k = 1; k < parts; k++) {
            CK(cudaEventRecord(g->ev_join[k - 1], g->pst[k - 1]));
            CK(cudaStreamWaitEvent(st, g->ev_join[k - 1], 0));
        }
        return WD_OK;
    }

    // stage s reads stage_src(s) and writes stage_dst(s): distinct arrays, because the stage
    // kernel of a far-field node re-evaluates its inner neighbours from the stage input
    T* stage_src(int s) { return s == 0 ? W(W_PHIN) : (s % 2 ? W(W_PHIS) : W(W_T0)); }
    T* stage_dst(int s) { return s % 2 ? W(W_T0) : W(W_PHIS); }

    wd_status step_part2d(F2Args<T, M>& a)
    {
        const PartTab<T> dt0 = g->dtab[0].template pview<T>(), dt1 = g->dtab[1].template pview<T>();
        bool merged_div = true;
        for (int s = 0; s < 4; s++) {
            a.src = stage_src(s);
            a.dst = stage_dst(s);
            a.stage = s;
            {
                // direction 1 first: the direction-0 pass combines both LAD terms and smooths
                // them along its lines
                ProfScope ps(g, WD_K_DERIV);
                CK(p2_launch<T, M>(a, dt1, F2_DERIV, 1, st));
                CK(p2_launch<T, M>(a, dt0, F2_DERIV, 0, st));
            }
            {
                ProfScope ps(g, WD_K_DIV);
                const cudaError_t e = merged_div ? p2_div2<T, M>(a, dt0, dt1, st) : cudaErrorNotSupported;
                if (e == cudaErrorNotSupported) {
                    cudaGetLastError();
                    merged_div = false;
                    CK(p2_launch<T, M>(a, dt0, F2_DIV, 0, st));
                    CK(p2_launch<T, M>(a, dt1, F2_DIV, 1, st));
                } else {
                    CK(e);
                }
            }
            {
                ProfScope ps(g, WD_K_POINT);
                CK(f2_launch<T, M>(a, F2_STAGE, st));
            }
        }
        a.src = stage_dst(3);
        a.dst = stage_dst(3);
        if (p->filter) {
            ProfScope ps(g, WD_K_FILTER);
            CK(p2_launch<T, M>(a, g->ftab[0].template pview<T>(), P2_FILTER0, 0, st));
        }
        ProfScope ps(g, WD_K_NORM);
        CK(p2_launch<T, M>(a, g->ftab[1].template pview<T>(), F2_FILTER, 1, st));
        return WD_OK;
    }

    wd_status step_fused(bool poisson)
    {
        if (p->filter) ST(ensure_filter(p->alpha_f));
        if (p->equation == WD_HJ_LAD && !poisson) ST(ensure_lads(p->lad_exp));
        F2Args<T, M> a = f2_args(poisson);
        if (p->filter) {
            LineOp op;
            ST(op_filter(p->alpha_f, op));
            std::memcpy(a.fa, op.fa, sizeof(a.fa));
        }
        if (line2d(a, poisson)) return step_line2d(poisson, line2d_parts());
        if (part2d(a)) return step_part2d(a);
        for (int s = 0; s < 4; s++) {
            a.src = stage_src(s);
            a.dst = stage_dst(s);
            a.stage = s;
            {
                ProfScope ps(g, WD_K_DERIV);
                CK(f2_launch<T, M>(a, F2_DERIV, st));
            }
            {
                ProfScope ps(g, WD_K_DIV);
                CK(f2_launch<T, M>(a, F2_DIV, st));
            }
            {
                ProfScope ps(g, WD_K_POINT);
                CK(f2_launch<T, M>(a, F2_STAGE, st));
            }
        }
        if (p->filter) ST(filter_dir(0, p->alpha_f, stage_dst(3), stage_dst(3)));
        a.src = stage_dst(3);
        ProfScope ps(g, WD_K_NORM);
        CK(f2_launch<T, M>(a, F2_FILTER, st));
        return WD_OK;
    }

    // uniform Cartesian 3-D grids with an explicit scheme and walls / periodic faces only
    // uniform Cartesian grids with an explicit scheme: 3-D with walls / periodic faces, or
    // single 2-D grids of any faces (far-field / Neumann faces are applied after each stage)
    bool cart3d() const
    {
        if (!g->cart || g->force_generic || g->batch != 1) return false;
        const int sch = g->desc.scheme;
        if (sch == WD_C4 || sch == WD_C6 || sch == WD_UW) return false;
        if (D.ndim == 2) return true;
        for (int d = 0; d < 3; d++)
            for (int k : {g->desc.bc_lo[d], g->desc.bc_hi[d]})
                if (k == WD_BC_FARFIELD || k == WD_BC_NEUMANN) return false;
        return true;
    }
    bool faces_need_bc() const
    {
        for (int d = 0; d < D.ndim; d++)
            for (int k : {g->desc.bc_lo[d], g->desc.bc_hi[d]})
                if (k == WD_BC_FARFIELD || k == WD_BC_NEUMANN) return true;
        return false;
    }

    C3Args<T> c3_args(bool poisson)
    {
        C3Args<T> a;
        std::memset(&a, 0, sizeof(a));
        a.D = D;
        a.scheme = g->desc.scheme;
        double s1 = 0.0, s2 = 0.0;
        for (int l = 0; l < D.ndim; l++) {
            a.ih[l] = T(1.0 / g->h[l]);
            a.slad[l] = T(std::pow(g->h[l], p->lad_exp - 4.0));
            s1 += 1.0 / g->h[l];
            s2 += 1.0 / (g->h[l] * g->h[l]);
        }
        a.sig1 = T(s1);
        a.sig2 = T(s2);
        a.phin = W(W_PHIN);
        a.acc = W(W_ACC);
        a.dtv = W(W_DT);
        a.U0 = W(W_U0);
        a.U1 = W(W_U1);
        a.U2 = W(W_U2);
        a.L = W(W_N0);
        a.G1 = W(W_N1);
        a.G2 = W(W_N2);
        a.mask = g->mask;
        a.dval = (const T*)g->dval;
        a.eps = T(p->eps);
        a.cfl = T(p->cfl);
        a.C_lad = T(p->C_lad);
        a.equation = p->equation;
        a.lad = p->equation == WD_HJ_LAD && !poisson;
        a.poisson = poisson;
        a.by = g->tune_by;
        a.vec = !g->line_off;
        return a;
    }

    // the line-resident filter passes of a uniform 3-D grid (directions 0 and 1): partition
    // tables along every direction, n0 a multiple of 32, the commit's partial sums in range
    bool line3_filters() const
    {
        if (D.ndim != 3 || g->line_off || g->part_off || D.n[0] % 32 != 0) return false;
        for (int d = 0; d < 3; d++) {
            const HostLineTab& t = p->filter ? g->ftab[d] : g->dtab[d];
            if (!t.pok) return false;
        }
        return (long long)D.nlines(2) / 32 <= g->npartial;
    }

    // the direction-2 filter with the commit streamed along z (wd_zfilter.cu)
    bool zfilter_ok() const
    {
        return p->filter && g->ztab && g->ztab_key == p->alpha_f && zfilter_supported(D, g->npartial);
    }
    ZfArgs<T> zf_args(bool poisson)
    {
        ZfArgs<T> z;
        std::memset(&z, 0, sizeof(z));
        z.D = D;
        z.src = W(W_PHIS);
        z.scratch = W(W_T0);
        z.phin = W(W_PHIN);
        z.phin_w = W(W_PHIN);
        z.mask = g->mask;
        z.dval = (const T*)g->dval;
        z.poisson = poisson;
        z.tab = (const T*)g->ztab;
        LineOp op;
        op_filter(p->alpha_f, op);
        for (int hw = 1; hw <= 5; hw++)
            for (int m = 1; m <= hw; m++) z.cf[hw][m] = T(0.5 * op.fa[hw][m] - (m == 1 ? p->alpha_f : 0.0));
        z.partial = g->partial;
        z.result = g->result;
        z.max_partials = g->npartial;
        return z;
    }

    // the partition pass that filters along direction 2 of a 3-D grid and commits
    F2Args<T, M> commit2_args(bool poisson)
    {
        F2Args<T, M> f;
        std::memset(&f, 0, sizeof(f));
        f.D = D;
        f.src = W(W_PHIS);
        f.dst = W(W_PHIS);
        f.phin = W(W_PHIN);
        f.phin_w = W(W_PHIN);
        f.mask = g->mask;
        f.dval = (const T*)g->dval;
        f.bclo1 = f.bchi1 = WD_BC_WALL;
        f.poisson = poisson;
        f.filter = 1;
        f.alpha_f = p->alpha_f;
        f.partial = g->partial;
        f.counter = g->counter;
        f.result = g->result;
        f.max_partials = g->npartial;
        f.batch = 1;
        LineOp op;
        op_filter(p->alpha_f, op);
        std::memcpy(f.fa, op.fa, sizeof(f.fa));
        return f;
    }

    wd_status step_cart3d(bool poisson)
    {
        if (p->filter) ST(ensure_filter(p->alpha_f));
        C3Args<T> a = c3_args(poisson);
        for (int s = 0; s < 4; s++) {
            a.src = s == 0 ? W(W_PHIN) : W(W_PHIS);
            a.dst = W(W_PHIS);
            a.stage = s;
            {
                ProfScope ps(g, WD_K_DERIV);
                CK(c3_launch<T>(a, C3_U, st));
            }
            if (a.lad) {
                ProfScope ps(g, WD_K_GAUSS);
                CK(c3_launch<T>(a, D.ndim == 3 ? C3_GXY : C3_GX, st));
            }
            {
                ProfScope ps(g, WD_K_POINT);
                CK(c3_launch<T>(a, C3_S, st));
            }
            if (faces_need_bc()) {
                if (D.ndim == 2) ST(bc_faces2d(W(W_PHIS), poisson));
                else ST(bc(W(W_PHIS), poisson));
            }
        }
        if (line3_filters() && p->filter) {
            // the line-resident filter passes along directions 0 (FX) and 1 (FY without
            // commit); the direction-2 filter with the commit stays on the partition pass below
            // (32-line blocks: a line-resident direction-2 commit measured 575 us against 245 us
            // on the 256^3 duct)
            L2Args<T, M> l = l2_args(poisson);
            l.kbeg = 0;
            l.kcnt = D.n[2];
            l.counter = g->counter;
            l.batch = 1;
            l.src = W(W_PHIS);
            l.dst = W(W_PHIS);
            {
                ProfScope ps(g, WD_K_FILTER);
                CK(l2_launch<T, M>(l, g->ftab[0].template pview<T>(), L2_FX, 2, st));
                l.commit = 0;
                l.fdir = 1;
                CK(l2_launch<T, M>(l, g->ftab[1].template pview<T>(), L2_FY, 2, st));
            }
            if (g->tune_zf && zfilter_ok()) {
                ProfScope ps(g, WD_K_NORM);
                CK(zfilter_commit<T>(zf_args(poisson), st));
                return WD_OK;
            }
            const F2Args<T, M> f = commit2_args(poisson);
            const PartTab<T> t2 = g->ftab[2].template pview<T>();
            if (p2_supported(f, t2, F2_FILTER, 2)) {
                ProfScope ps(g, WD_K_NORM);
                CK(p2_launch<T, M>(f, t2, F2_FILTER, 2, st));
                return WD_OK;
            }
            ST(filter_dir(2, p->alpha_f, W(W_PHIS), W(W_PHIS)));
            ST(bc(W(W_PHIS), poisson));
            ProfScope ps(g, WD_K_NORM);
            CK(launch_norms<T>(D, W(W_PHIS), W(W_PHIN), g->mask, g->partial, g->counter, g->result,
                               g->nred, st));
            return WD_OK;
        }
        // filter along 0, 1 and 2 with the warp partition passes; the direction-2 pass also
        // resets the Dirichlet nodes, reduces the change norms and commits
        F2Args<T, M> f;
        std::memset(&f, 0, sizeof(f));
        f.D = D;
        f.src = W(W_PHIS);
        f.dst = W(W_PHIS);
        f.phin = W(W_PHIN);
        f.phin_w = W(W_PHIN);
        f.mask = g->mask;
        f.dval = (const T*)g->dval;
        f.bclo1 = f.bchi1 = WD_BC_WALL;
        f.poisson = poisson;
        f.filter = p->filter;
        f.alpha_f = p->alpha_f;
        f.partial = g->partial;
        f.counter = g->counter;
        f.result = g->result;
        f.max_partials = g->npartial;
        f.batch = 1;
        bool part = !g->part_off && D.ndim == 3;
        if (p->filter) {
            LineOp op;
            ST(op_filter(p->alpha_f, op));
            std::memcpy(f.fa, op.fa, sizeof(f.fa));
        }
        for (int d = 0; d < 3 && part; d++) {
            const PartTab<T> ft = g->ftab[d].template pview<T>();
            if (p->filter ? !p2_supported(f, ft, d == 2 ? F2_FILTER : P2_FILTER0, d)
                          : (d == 2 && !p2_supported(f, g->dtab[2].template pview<T>(), F2_FILTER, d)))
                part = false;
        }
        if (part) {
            if (p->filter) {
                ProfScope ps(g, WD_K_FILTER);
                for (int d = 0; d < 2; d++)
                    CK(p2_launch<T, M>(f, g->ftab[d].template pview<T>(), P2_FILTER0, d, st));
            }
            ProfScope ps(g, WD_K_NORM);
            const PartTab<T> t2 = p->filter ? g->ftab[2].template pview<T>() : g->dtab[2].template pview<T>();
            CK(p2_launch<T, M>(f, t2, F2_FILTER, 2, st));
            return WD_OK;
        }
        if (p->filter) {
            for (int d = 0; d < D.ndim; d++) {
                const PartTab<T> ft = g->ftab[d].template pview<T>();
                if (!g->part_off && p2_supported(f, ft, P2_FILTER0, d)) {
                    ProfScope ps(g, WD_K_FILTER);
                    CK(p2_launch<T, M>(f, ft, P2_FILTER0, d, st));
                } else {
                    ST(filter_dir(d, p->alpha_f, W(W_PHIS), W(W_PHIS)));
                }
            }
            ST(bc(W(W_PHIS), poisson));
        }
        ProfScope ps(g, WD_K_NORM);
        CK(launch_norms<T>(D, W(W_PHIS), W(W_PHIN), g->mask, g->partial, g->counter, g->result,
                           g->nred, st));
        return WD_OK;
    }

    // one pseudo step from W_PHIN; leaves the new state in W_PHIN and the change norms in
    // g->result
    wd_status step(bool poisson)
    {
        if (fused2d()) return step_fused(poisson);
        if (cart3d() && !(p->curvature && !poisson)) return step_cart3d(poisson);
        if (g->batch > 1) return set_error(WD_ERR_INVALID_ARG, "stacked 2-D grids need the fused path");
        for (int s = 0; s < 4; s++) {
            const T* src = s == 0 ? W(W_PHIN) : W(W_PHIS);
            ST(rhs_into(src, W(W_PHIS), poisson, s));
            ST(bc(W(W_PHIS), poisson));
        }
        if (p->filter) {
            for (int d = 0; d < D.ndim; d++) ST(filter_dir(d, p->alpha_f, W(W_PHIS), W(W_PHIS)));
            ST(bc(W(W_PHIS), poisson));
        }
        ProfScope ps(g, WD_K_NORM);
        CK(launch_norms<T>(D, W(W_PHIS), W(W_PHIN), g->mask, g->partial, g->counter, g->result,
                           g->nred, st));
        return WD_OK;
    }

    // Runs n pseudo steps.  Without the kernel timer the steps are captured once into a
    // CUDA graph (n steps per graph) and replayed, so the launch sequence costs one graph
    // launch per n steps.  The graph stays with the grid and is reused by later solves with
    // the same n and parameters; the first step of a solve phase runs uncaptured so that
    // every table and kernel attribute exists before a capture.
    wd_status run_steps(bool poisson, int n, bool& warmed)
    {
        if (n <= 0) return WD_OK;
        if (g->prof_on || !warmed) {
            for (int i = 0; i < n; i++) ST(step(poisson));
            warmed = true;
            return WD_OK;
        }
        const int k = poisson ? 1 : 0;
        const bool hit = g->gx[k] && g->gx_n[k] == n && g->gx_gen[k] == g->gen &&
                         std::memcmp(&g->gx_p[k], p, sizeof(*p)) == 0;
        if (!hit) {
            if (g->gx[k]) cudaGraphExecDestroy(g->gx[k]);
            g->gx[k] = nullptr;
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            wd_status rs = WD_OK;
            for (int i = 0; i < n && rs == WD_OK; i++) rs = step(poisson);
            cudaError_t ce = cudaStreamEndCapture(st, &graph);
            if (rs != WD_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rs;
            }
            CK(ce);
            cudaGraphExec_t ex = nullptr;
            ce = cudaGraphInstantiate(&ex, graph, 0);
            cudaGraphDestroy(graph);
            CK(ce);
            g->gx[k] = ex;
            g->gx_n[k] = n;
            g->gx_gen[k] = g->gen;
            g->gx_p[k] = *p;
        }
        CK(cudaGraphLaunch(g->gx[k], st));
        return WD_OK;
    }

    // change norms of the last pseudo step; stacked grids report their worst member
    cudaError_t enqueue_norms()
    {
        return cudaMemcpyAsync(g->hres, g->result, (size_t)2 * g->batch * sizeof(double),
                               cudaMemcpyDeviceToHost, st);
    }
    void eval_norms(double scale, double* l2, double* linf) const
    {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < g->batch; k++) {
            const double n = g->nact[k] > 0 ? (double)g->nact[k] : 1.0;
            const double l = std::sqrt(g->hres[2 * k] / n) / scale;
            const double m = g->hres[2 * k + 1] / scale;
            if (!(l <= a)) a = l;   // keeps NaN
            if (!(m <= b)) b = m;
        }
        *l2 = a;
        *linf = b;
    }
    wd_status read_norms(double scale, double* l2, double* linf)
    {
        CK(enqueue_norms());
        CK(cudaStreamSynchronize(st));
        eval_norms(scale, l2, linf);
        return WD_OK;
    }

    wd_status spalding_from_phin()
    {
        ST(grad_parts(W(W_PHIN), false));
        T* U[3] = {W(W_U0), W(W_U1), W(W_U2)};
        CK(launch_spalding<T, M>(D, U, W(W_PHIN), W(W_PHIN), st));
        return WD_OK;
    }

    // ---- a solve as a resumable task ------------------------------------------------
    // begin() enqueues the initial state; each enqueue() queues one slice of pseudo steps
    // that ends at a convergence check (every check_every steps) together with the copy of
    // its change norms; complete(), called once that slice has finished on the device,
    // evaluates the norms and advances the state; finish() queues the copy-out.  solve()
    // runs the same sequence synchronously, so a solve gives identical results whether it
    // runs alone or interleaved with others.
    struct Run {
        int phase = 0;                 // 0 Poisson guess, 1 HJ marching, 2 finished
        int it = 0, pit = 0, every = 1;
        bool warmed = false, check = false, have_tol = false;
        double l2 = 0.0, li = 0.0, best = INFINITY;
        int since_best = 0;
        wd_stats s;
        wd_status rc = WD_OK;
    } R;

    wd_status enter_hj(bool after_poisson)
    {
        if (after_poisson) ST(spalding_from_phin());
        ST(bc(W(W_PHIN), false));
        R.phase = p->max_iters > 0 ? 1 : 2;
        R.warmed = false;
        return WD_OK;
    }

    // times the free launch shapes of this grid's path once (see the autotuner above); stage
    // 0 of every timed kernel overwrites its outputs, and the first pseudo step recomputes them
    wd_status autotune()
    {
        if (g->tuned || g->prof_on || !autotune_enabled()) return WD_OK;
        g->tuned = 1;
        char key[160];
        std::snprintf(key, sizeof(key), "%d:%dx%dx%d:p%d:s%d:e%d:c%d:%s", D.ndim, D.n[0], D.n[1], D.n[2],
                      g->desc.precision, g->desc.scheme, p->equation, p->curvature,
                      fused2d() ? "f2" : (cart3d() ? "c3" : "gen"));
        if (fused2d() && g->batch > 1 && g->ev_fork) {
            if (p->filter) ST(ensure_filter(p->alpha_f));
            if (p->equation == WD_HJ_LAD) ST(ensure_lads(p->lad_exp));
            F2Args<T, M> f = f2_args(false);
            if (line2d(f, false)) {
                // parts of the batch: one pseudo step's worth of the passes of stage 0 (they
                // overwrite their outputs; the first real step recomputes them from phi^n)
                std::string k2 = std::string(key) + ":l2parts";
                g->tune_parts = tune_choice(k2, {1, 2, 4}, [&](int c) {
                    if (c > g->batch) return 1e30f;
                    return time_calls(st, [&] { step_line2d(false, c); });
                });
            }
        }
        if (fused2d()) {
            if (p->equation == WD_HJ_LAD) ST(ensure_lads(p->lad_exp));
            F2Args<T, M> a = f2_args(false);
            a.src = W(W_PHIN);
            a.dst = W(W_PHIS);
            a.stage = 0;
            g->tune_stage_threads = tune_choice(key, {128, 256, 512}, [&](int c) {
                a.stage_threads = c;
                return time_calls(st, [&] { f2_launch<T, M>(a, F2_STAGE, st); });
            });
        } else if (cart3d()) {
            C3Args<T> a = c3_args(false);
            a.src = W(W_PHIN);
            a.dst = W(W_PHIS);
            a.stage = 0;
            g->tune_by = tune_choice(key, {4, 8, 16}, [&](int c) {
                a.by = c;
                return time_calls(st, [&] {
                    c3_launch<T>(a, C3_U, st);
                    c3_launch<T>(a, C3_S, st);
                });
            });
            if (p->filter && line3_filters()) {
                // the direction-2 filter + commit: streamed along z (1) or the partition pass
                // (0); both overwrite phi^n, which begin() sets after this
                ST(ensure_filter(p->alpha_f));
                const F2Args<T, M> f = commit2_args(false);
                const PartTab<T> t2 = g->ftab[2].template pview<T>();
                if (zfilter_ok() && p2_supported(f, t2, F2_FILTER, 2))
                    g->tune_zf = tune_choice(std::string(key) + ":zf", {1, 0}, [&](int c) {
                        if (c) return time_calls(st, [&] { zfilter_commit<T>(zf_args(false), st); });
                        return time_calls(st, [&] { p2_launch<T, M>(f, t2, F2_FILTER, 2, st); });
                    });
            }
        }
        CK(cudaGetLastError());
        return WD_OK;
    }

    wd_status begin(const void* phi_user, bool warm)
    {
        ST(autotune());
        R = Run();
        std::memset(&R.s, 0, sizeof(R.s));
        R.every = p->check_every > 0 ? p->check_every : 1;
        R.have_tol = p->tol_l2 > 0.0 || p->tol_linf > 0.0;
        const int init = warm ? WD_INIT_GIVEN : p->init;
        if (init == WD_INIT_GIVEN) {
            CK(to_padded(g, W(W_PHIN), phi_user, sizeof(T)));
        } else {
            CK(launch_fill<T>(W(W_PHIN), D.total, T(0), st));
        }
        if (init == WD_INIT_POISSON && p->poisson_max_iters > 0) {
            ST(bc(W(W_PHIN), true));
            R.phase = 0;
            return WD_OK;
        }
        return enter_hj(init == WD_INIT_POISSON);
    }

    bool finished() const { return R.phase >= 2; }
    int stall_window() const
    {
        int w = 200;
        for (int d = 0; d < D.ndim; d++) w = std::max(w, 2 * D.n[d]);
        return w;
    }

    wd_status enqueue()
    {
        if (R.phase == 0) {
            const int n = std::min(R.every - R.pit % R.every, p->poisson_max_iters - R.pit);
            ST(run_steps(true, n, R.warmed));
            R.pit += n;
            R.check = p->poisson_tol > 0.0 && R.pit % R.every == 0;
        } else if (R.phase == 1) {
            const int n = std::min(R.every - R.it % R.every, p->max_iters - R.it);
            ST(run_steps(false, n, R.warmed));
            R.it += n;
            R.check = true;     // every slice ends on a multiple of check_every or at max_iters
        } else {
            R.check = false;
        }
        if (R.check) CK(enqueue_norms());
        return WD_OK;
    }

    wd_status complete()
    {
        const double L = g->desc.L_ref;
        if (R.phase == 0) {
            bool done = R.pit >= p->poisson_max_iters;
            if (R.check) {
                double l2, li;
                eval_norms(L * L, &l2, &li);
                if (!std::isfinite(l2) || !std::isfinite(li) || l2 <= p->poisson_tol) done = true;
            }
            if (done) {
                R.s.poisson_iters = R.pit;
                ST(enter_hj(true));
            }
            return WD_OK;
        }
        if (R.phase != 1) return WD_OK;
        eval_norms(L, &R.l2, &R.li);
        if (!std::isfinite(R.l2) || !std::isfinite(R.li)) {
            R.s.diverged = 1;
            R.rc = WD_ERR_DIVERGED;
            R.phase = 2;
            return WD_OK;
        }
        if (R.have_tol && (p->tol_l2 <= 0.0 || R.l2 <= p->tol_l2) &&
            (p->tol_linf <= 0.0 || R.li <= p->tol_linf)) {
            R.s.converged = 1;
            R.phase = 2;
            return WD_OK;
        }
        if (R.l2 < 0.95 * R.best) {
            R.best = R.l2;
            R.since_best = 0;
        } else {
            R.since_best += R.every;
        }
        // FP32 state: the change norm stops falling at the round-off floor; stop when the
        // best RMS change has not improved by 5 % over a window long enough for a front to
        // cross the grid twice (at most one node per pseudo step): max(200, 2 max_l n_l)
        if (sizeof(T) == 4 && R.have_tol && R.since_best >= stall_window()) {
            R.s.converged = 1;
            R.s.stalled = 1;
            R.phase = 2;
            return WD_OK;
        }
        if (R.it >= p->max_iters) R.phase = 2;
        return WD_OK;
    }

    // queues the copy of the result into phi_user; the stats are final once it has run
    wd_status finish(void* phi_user, wd_stats* stats)
    {
        wd_status rc = R.rc;
        if (rc == WD_OK && R.have_tol && !R.s.converged) rc = WD_ERR_NOT_CONVERGED;
        R.s.iters = R.it;
        R.s.res_l2 = R.l2;
        R.s.res_linf = R.li;
        R.s.device_bytes = g->bytes;
        CK(from_padded(g, phi_user, W(W_PHIN), sizeof(T)));
        if (stats) *stats = R.s;
        if (rc == WD_ERR_DIVERGED) set_error(rc, "non-finite pseudo-step change");
        if (rc == WD_ERR_NOT_CONVERGED) set_error(rc, "max_iters reached before the tolerance");
        return rc;
    }

    // full solve; phi_user is read for WD_INIT_GIVEN (or warm) and receives the result
    wd_status solve(void* phi_user, wd_stats* stats, bool warm)
    {
        ST(begin(phi_user, warm));
        while (!finished()) {
            ST(enqueue());
            if (R.check) CK(cudaStreamSynchronize(st));
            ST(complete());
        }
        wd_status rc = finish(phi_user, stats);
        CK(cudaStreamSynchronize(st));
        return rc;
    }

    wd_status steps(int kind, void* phi_user, int n, wd_stats* stats)
    {
        bool poisson = kind == 1;
        double scale = poisson ? g->desc.L_ref * g->desc.L_ref : g->desc.L_ref;
        CK(to_padded(g, W(W_PHIN), phi_user, sizeof(T)));
        for (int i = 0; i < n; i++) ST(step(poisson));
        double l2 = 0, li = 0;
        if (n > 0) ST(read_norms(scale, &l2, &li));
        CK(from_padded(g, phi_user, W(W_PHIN), sizeof(T)));
        CK(cudaStreamSynchronize(st));
        if (stats) {
            std::memset(stats, 0, sizeof(*stats));
            if (poisson) stats->poisson_iters = n;
            else stats->iters = n;
            stats->res_l2 = l2;
            stats->res_linf = li;
            stats->diverged = !(std::isfinite(l2) && std::isfinite(li));
            stats->device_bytes = g->bytes;
        }
        return WD_OK;
    }

    UwCart<M> uw_cart() const
    {
        UwCart<M> c;
        c.cart = g->cart;
        for (int l = 0; l < 3; l++) c.ih[l] = g->cart && l < D.ndim ? M(1.0 / g->h[l]) : M(0);
        return c;
    }

    // one step of the level-set equation (Sec. 5.5) from a to b: four stage kernels whose
    // outputs never alias their inputs (a -> T0 -> T1 -> T0 -> b, phin = a)
    wd_status ls_step(T* a, T* b, double F, double dt)
    {
        LsArgs<T, M> x;
        x.phin = a;
        x.acc = W(W_ACC);
        x.xi = xi();
        x.cc = uw_cart();
        x.F = F;
        x.dt = dt;
        T* io[5] = {a, W(W_T0), W(W_T1), W(W_T0), b};
        for (int k = 0; k < 4; k++) {
            x.src = io[k];
            x.dst = io[k + 1];
            ProfScope ps(g, WD_K_POINT);
            CK(launch_ls_stage<T, M>(D, x, k, st));
        }
        return WD_OK;
    }

    // n level-set steps; the state alternates between W_PHIN and W_PHIS.  Pairs of steps
    // (PHIN -> PHIS -> PHIN) run as one CUDA graph, captured after a first uncaptured pair
    // and kept with the grid for the same F and dt.
    wd_status levelset(void* phi_user, double F, double dt, int n)
    {
        CK(to_padded(g, W(W_PHIN), phi_user, sizeof(T)));
        T* a = W(W_PHIN);
        T* b = W(W_PHIS);
        int pairs = n / 2;
        const bool hit = g->lsx && g->ls_F == F && g->ls_dt == dt && g->ls_gen == g->gen;
        if (pairs > 0 && (g->prof_on || !hit)) {
            ST(ls_step(a, b, F, dt));
            ST(ls_step(b, a, F, dt));
            pairs--;
            if (g->prof_on) {
                for (; pairs > 0; pairs--) {
                    ST(ls_step(a, b, F, dt));
                    ST(ls_step(b, a, F, dt));
                }
            } else if (pairs > 0) {
                if (g->lsx) cudaGraphExecDestroy(g->lsx);
                g->lsx = nullptr;
                cudaGraph_t graph = nullptr;
                CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                wd_status rs = ls_step(a, b, F, dt);
                if (rs == WD_OK) rs = ls_step(b, a, F, dt);
                cudaError_t ce = cudaStreamEndCapture(st, &graph);
                if (rs != WD_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return rs;
                }
                CK(ce);
                cudaGraphExec_t ex = nullptr;
                ce = cudaGraphInstantiate(&ex, graph, 0);
                cudaGraphDestroy(graph);
                CK(ce);
                g->lsx = ex;
                g->ls_F = F;
                g->ls_dt = dt;
                g->ls_gen = g->gen;
            }
        }
        for (; pairs > 0; pairs--) CK(cudaGraphLaunch(g->lsx, st));
        if (n % 2) {
            ST(ls_step(a, b, F, dt));
            std::swap(a, b);
        }
        CK(from_padded(g, phi_user, a, sizeof(T)));
        CK(cudaStreamSynchronize(st));
        return WD_OK;
    }

    wd_status rhs(int kind, const void* phi_user, void* R_user, void* dt_user)
    {
        bool poisson = kind == 1;
        CK(to_padded(g, W(W_PHIN), phi_user, sizeof(T)));
        ST(rhs_into(W(W_PHIN), W(W_PHIS), poisson, -1));
        if (R_user) CK(from_padded(g, R_user, W(W_PHIS), sizeof(T)));
        if (dt_user) CK(from_padded(g, dt_user, W(W_DT), sizeof(T)));
        return WD_OK;
    }
};

template <typename F>
static wd_status dispatch(wd_grid g, F&& fn)
{
    switch (g->desc.precision) {
    case WD_FP64: {
        auto r = fn((double*)nullptr, (double*)nullptr);
        return r;
    }
    default: return fn((float*)nullptr, (float*)nullptr);
    }
}

// ------------------------------------------------------------------------------------
// grid creation
// ------------------------------------------------------------------------------------

// device arrays whose size and contents depend on the descriptor only
template <typename T, typename M>
static wd_status alloc_impl(wd_grid g)
{
    const Dims& D = g->D;
    cudaStream_t st = g->stream;
    const long long tot = D.total;
    ST(dmalloc(g, (void**)&g->xyz, (size_t)tot * 3 * 8));
    CK(cudaMemsetAsync(g->xyz, 0, (size_t)tot * 3 * 8, st));
    // line tables
    for (int d = 0; d < D.ndim; d++) {
        std::vector<double> a, c;
        int imp;
        derivative_rows(central_scheme(g->desc.scheme), D.n[d], D.per[d], a, c, imp);
        ST(build_line_table(D.n[d], D.per[d], a, c, imp, g->dtab[d]));
        std::vector<double> z(D.n[d], 0.0);
        ST(build_line_table(D.n[d], D.per[d], z, z, 0, g->etab[d]));
    }
    ST(dmalloc(g, (void**)&g->xi_d, (size_t)tot * 9 * 8));
    ST(dmalloc(g, (void**)&g->J_d, (size_t)tot * 8));
    ST(dmalloc(g, (void**)&g->dx_d, (size_t)tot * 3 * 8));
    CK(cudaMemsetAsync(g->xi_d, 0, (size_t)tot * 9 * 8, st));
    CK(cudaMemsetAsync(g->dx_d, 0, (size_t)tot * 3 * 8, st));
    if (sizeof(M) == 8) {
        g->xi_m = g->xi_d;
        g->xi_alias = 1;
    } else {
        ST(dmalloc(g, &g->xi_m, (size_t)tot * 9 * sizeof(M)));
        CK(cudaMemsetAsync(g->xi_m, 0, (size_t)tot * 9 * sizeof(M), st));
        g->xi_alias = 0;
    }
    ST(dmalloc(g, &g->sig1, (size_t)tot * sizeof(M)));
    ST(dmalloc(g, &g->sig2, (size_t)tot * sizeof(M)));
    ST(dmalloc(g, &g->lads, (size_t)tot * 3 * sizeof(M)));
    long long fmax = 0;
    for (int d = 0; d < 3; d++) {
        long long f = (long long)D.n[(d + 1) % 3] * D.n[(d + 2) % 3];
        if (f > fmax) fmax = f;
    }
    g->fmax = fmax;
    ST(dmalloc(g, (void**)&g->ffr, (size_t)fmax * 6 * 8));
    CK(cudaMemsetAsync(g->ffr, 0, (size_t)fmax * 6 * 8, st));
    // wall faces (Dirichlet 0)
    ST(dmalloc(g, (void**)&g->wall, (size_t)tot));
    ST(dmalloc(g, (void**)&g->mask, (size_t)tot));
    ST(dmalloc(g, &g->dval, (size_t)tot * sizeof(T)));
    {
        std::vector<uint8_t> wall((size_t)tot, 0);
        for (int k = 0; k < D.n[2]; k++)
            for (int j = 0; j < D.n[1]; j++)
                for (int i = 0; i < D.n[0]; i++) {
                    int c[3] = {i, j, k};
                    bool w = false;
                    for (int d = 0; d < D.ndim; d++) {
                        if (c[d] == 0 && g->desc.bc_lo[d] == WD_BC_WALL) w = true;
                        if (c[d] == D.n[d] - 1 && g->desc.bc_hi[d] == WD_BC_WALL) w = true;
                    }
                    wall[(size_t)D.idx(i, j, k)] = w;
                }
        CK(cudaMemcpyAsync(g->wall, wall.data(), (size_t)tot, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    ST(dmalloc(g, (void**)&g->dcount, sizeof(unsigned long long)));
    for (int k = 0; k < W_NWORK; k++) {
        if (k == W_ADV && g->desc.scheme != WD_UW) continue;   // the upwind term: baseline only
        ST(dmalloc(g, &g->w[k], (size_t)tot * sizeof(T)));
        CK(cudaMemsetAsync(g->w[k], 0, (size_t)tot * sizeof(T), st));
    }
    g->nred = (int)std::min<long long>((tot + 255) / 256, 1024);
    g->npartial = std::max(g->nred, D.n[0] * D.n[2]);
    ST(dmalloc(g, (void**)&g->partial, (size_t)g->npartial * 2 * 8));
    ST(dmalloc(g, (void**)&g->counter, wd_grid_s::NPART * sizeof(unsigned)));
    ST(dmalloc(g, (void**)&g->result, (size_t)2 * g->batch * 8));
    CK(cudaMemsetAsync(g->counter, 0, (size_t)wd_grid_s::NPART * sizeof(unsigned), st));
    CK(cudaMemsetAsync(g->result, 0, (size_t)2 * g->batch * 8, st));
    if (cudaMallocHost(&g->hres, (size_t)2 * g->batch * sizeof(double)) != cudaSuccess)
        return set_error(WD_ERR_OOM, "pinned");
    CK(cudaStreamSynchronize(st));
    return WD_OK;
}

// coordinates, metrics (Sec. 3.1), far-field spacing ratios and the Dirichlet set; temporary
// device memory comes from the stream-ordered allocator, so nothing here waits for other
// streams
template <typename T, typename M>
static wd_status geometry_impl(wd_grid g, const double* xyz_host, const uint8_t* mask_host,
                               const double* dval_host)
{
    const Dims& D = g->D;
    cudaStream_t st = g->stream;
    const long long tot = D.total;
    g->gen++;
    g->lads_exp = -1.0;
    for (int m = 0; m < D.ndim; m++)
        CK(cudaMemcpy2DAsync(g->xyz + m * tot, (size_t)D.pitch * 8,
                             xyz_host + (size_t)m * D.n[0] * D.n[1] * D.n[2], (size_t)D.n[0] * 8,
                             (size_t)D.n[0] * 8, (size_t)D.n[1] * D.n[2], cudaMemcpyHostToDevice, st));
    // uniform Cartesian grid?  x = x0 + i hx, y = y0 + j hy (, z = z0 + k hz) at every node
    g->cart = 0;
    if (D.ndim == 3 || g->batch == 1) {
        const bool d3 = D.ndim == 3;
        const size_t N = (size_t)D.n[0] * D.n[1] * D.n[2];
        const double* X = xyz_host;
        const double* Y = xyz_host + N;
        const size_t s1 = D.n[0], s2 = (size_t)D.n[0] * D.n[1];
        std::vector<double> zero;
        if (!d3) zero.assign(N, 0.0);
        const double* Z = d3 ? xyz_host + 2 * N : zero.data();
        double hx = X[1] - X[0], hy = Y[s1] - Y[0], hz = d3 ? Z[s2] - Z[0] : 1.0;
        bool ok = hx > 0 && hy > 0 && hz > 0;
        const double tx = 1e-9 * (std::fabs(X[0]) + D.n[0] * hx), ty = 1e-9 * (std::fabs(Y[0]) + D.n[1] * hy),
                     tz = 1e-9 * (std::fabs(Z[0]) + D.n[2] * hz);
        for (int k = 0; k < D.n[2] && ok; k++)
            for (int j = 0; j < D.n[1] && ok; j++)
                for (int i = 0; i < D.n[0]; i++) {
                    const size_t q = i + s1 * j + s2 * k;
                    if (std::fabs(X[q] - (X[0] + i * hx)) > tx || std::fabs(Y[q] - (Y[0] + j * hy)) > ty ||
                        (d3 && std::fabs(Z[q] - (Z[0] + k * hz)) > tz)) {
                        ok = false;
                        break;
                    }
                }
        g->cart = ok;
        g->h[0] = hx;
        g->h[1] = hy;
        g->h[2] = hz;
    }
    // metrics: A[(m*3+l)] = dx_m/dxi_l by the grid's scheme, periodic shift added back
    {
        double* A = nullptr;
        double* tmp = nullptr;
        if (cudaMallocAsync((void**)&A, (size_t)tot * 9 * 8, st) != cudaSuccess ||
            cudaMallocAsync((void**)&tmp, (size_t)tot * 8, st) != cudaSuccess) {
            if (A) cudaFreeAsync(A, st);
            cudaGetLastError();
            return set_error(WD_ERR_OOM, "metric scratch");
        }
        // WD_FP32: the coordinates are rounded to FP32 and differentiated in FP32
        const bool f32 = g->desc.precision == WD_FP32;
        float* fx = nullptr;
        if (f32 && cudaMallocAsync((void**)&fx, (size_t)tot * 2 * sizeof(float), st) != cudaSuccess) {
            cudaFreeAsync(A, st);
            cudaFreeAsync(tmp, st);
            cudaGetLastError();
            return set_error(WD_ERR_OOM, "metric scratch");
        }
        cudaError_t ce = cudaSuccess;
        LineOp op;
        std::memset(&op, 0, sizeof(op));
        op.kind = OPK_DERIV;
        op.scheme = central_scheme(g->desc.scheme);
        for (int l = 0; l < D.ndim && ce == cudaSuccess; l++)
            for (int m = 0; m < D.ndim && ce == cudaSuccess; m++) {
                double shift = D.per[l] ? g->desc.period[l][m] : 0.0;
                const double* src = g->xyz + m * tot;
                if (shift != 0.0) {
                    ce = launch_unwrap(D, l, src, shift, tmp, st);
                    src = tmp;
                }
                double* out = A + (long long)(m * 3 + l) * tot;
                if (f32) {
                    Fields<float> f;
                    std::memset(&f, 0, sizeof(f));
                    f.in[0] = fx;
                    f.out[0] = fx + tot;
                    if (ce == cudaSuccess) ce = launch_convert<double, float>(src, fx, tot, st);
                    if (ce == cudaSuccess)
                        ce = launch_line<float, float>(D, l, g->dtab[l], op, 1, 0, f, nullptr, 0, 0, st);
                    if (ce == cudaSuccess) ce = launch_convert<float, double>(fx + tot, out, tot, st);
                } else {
                    Fields<double> f;
                    std::memset(&f, 0, sizeof(f));
                    f.in[0] = src;
                    f.out[0] = out;
                    if (ce == cudaSuccess)
                        ce = launch_line<double, double>(D, l, g->dtab[l], op, 1, 0, f, nullptr, 0, 0, st);
                }
                // derivative of the removed linear part shift * t / n: shift / n, exact for
                // every scheme
                if (ce == cudaSuccess && shift != 0.0)
                    ce = launch_add_const(D, A + (long long)(m * 3 + l) * tot, shift / D.n[l], st);
            }
        if (ce == cudaSuccess)
            ce = launch_metric_finish<M>(D, A, g->xi_d, g->J_d, g->dx_d,
                                         g->xi_alias ? nullptr : (M*)g->xi_m, (M*)g->sig1, (M*)g->sig2, st);
        cudaFreeAsync(A, st);
        cudaFreeAsync(tmp, st);
        if (fx) cudaFreeAsync(fx, st);
        if (ce != cudaSuccess) return cuda_error(ce, "metrics");
    }
    CK(launch_ff_ratio(D, g->xyz, g->ffr, g->fmax, st));
    // Dirichlet set: wall faces + caller mask
    {
        uint8_t* um = nullptr;
        T* uv = nullptr;
        const size_t Nd = (size_t)D.n[0] * D.n[1] * D.n[2];
        if (mask_host) {
            if (cudaMallocAsync((void**)&um, Nd, st) != cudaSuccess) {
                cudaGetLastError();
                return set_error(WD_ERR_OOM, "mask upload");
            }
            CK(cudaMemcpyAsync(um, mask_host, Nd, cudaMemcpyHostToDevice, st));
            if (dval_host) {
                std::vector<T> v(Nd);
                for (size_t q = 0; q < Nd; q++) v[q] = (T)dval_host[q];
                if (cudaMallocAsync((void**)&uv, Nd * sizeof(T), st) != cudaSuccess) {
                    cudaFreeAsync(um, st);
                    cudaGetLastError();
                    return set_error(WD_ERR_OOM, "dval upload");
                }
                // the staging copy of pageable memory completes before the call returns
                CK(cudaMemcpyAsync(uv, v.data(), Nd * sizeof(T), cudaMemcpyHostToDevice, st));
            }
        }
        cudaError_t ce = launch_mask_merge<T>(D, um, uv, g->mask, (T*)g->dval, g->wall, st);
        if (um) cudaFreeAsync(um, st);
        if (uv) cudaFreeAsync(uv, st);
        if (ce != cudaSuccess) return cuda_error(ce, "mask merge");
    }
    return WD_OK;
}

static wd_status count_active(wd_grid g)
{
    // stacked 2-D grids are contiguous blocks of pitch * n[1] elements
    Dims one = g->D;
    const int B = g->batch;
    if (B > 1) {
        one.n[2] = 1;
        one.total = (long long)one.pitch * one.n[1];
    }
    g->nact.assign(B, 0);
    g->nactive = 0;
    for (int k = 0; k < B; k++) {
        CK(cudaMemsetAsync(g->dcount, 0, sizeof(unsigned long long), g->stream));
        CK(launch_count(one, g->mask + (long long)k * one.total, g->dcount, g->stream));
        unsigned long long c = 0;
        CK(cudaMemcpyAsync(&c, g->dcount, sizeof(c), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        g->nact[k] = (long long)c;
        g->nactive += (long long)c;
    }
    return WD_OK;
}

extern "C" {

void wd_default_params(int scheme, wd_solve_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->equation = WD_HJ_LAD;
    p->curvature = 0;
    p->eps = 0.2;
    p->C_lad = 0.1;
    p->lad_exp = 3.0;
    p->alpha_f = 0.49;
    p->filter = scheme == WD_UW ? 0 : 1;     // the baseline's upwinding damps by itself
    p->cfl = (scheme == WD_C4 || scheme == WD_C6) ? 0.6 : 0.8;
    p->eps0 = 1e-8;
    p->tol_l2 = 1e-10;
    p->tol_linf = 0.0;
    p->max_iters = 20000;
    p->check_every = 10;
    p->init = WD_INIT_POISSON;
    p->poisson_tol = 0.0;
    p->poisson_max_iters = 100;
}

wd_status wd_create_grid(const wd_grid_desc* desc, const double* xyz_host, const uint8_t* mask_host,
                         const double* dval_host, void* cuda_stream, wd_grid* out)
{
    if (!out) return set_error(WD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ST(validate_desc(desc));
    if (!xyz_host) return set_error(WD_ERR_INVALID_ARG, "xyz_host is NULL");
    wd_grid g = new wd_grid_s();
    g->desc = *desc;
    g->user_stream = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        release(g);
        return cuda_error(e, "stream / event creation");
    }
    if (desc->ndim == 2 && desc->n[2] > 1) {
        bool ok = cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < wd_grid_s::NPART - 1; k++)
            ok = cudaStreamCreateWithFlags(&g->pst[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&g->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaError_t e = cudaGetLastError();
            release(g);
            return cuda_error(e, "stream / event creation");
        }
    }
    g->es = desc->precision == WD_FP64 ? 8 : 4;
    Dims& D = g->D;
    D.ndim = desc->ndim;
    for (int k = 0; k < 3; k++) {
        D.n[k] = desc->n[k];
        D.per[k] = k < desc->ndim && desc->bc_lo[k] == WD_BC_PERIODIC;
    }
    D.pitch = (desc->n[0] + 31) / 32 * 32;
    D.total = (long long)D.pitch * D.n[1] * D.n[2];
    g->batch = desc->ndim == 2 ? desc->n[2] : 1;
    {
        const char* fg = std::getenv("WD_FORCE_GENERIC");
        g->force_generic = fg && fg[0] == '1';
        const char* po = std::getenv("WD_PART_OFF");
        g->part_off = po && po[0] == '1';
        const char* lo = std::getenv("WD_LINE2D_OFF");
        g->line_off = lo && lo[0] == '1';
    }
    wd_status s;
    {
        StreamGuard sg(g);
        s = dispatch(g, [&](auto* t, auto* m) {
            using T = std::remove_pointer_t<decltype(t)>;
            using M = std::remove_pointer_t<decltype(m)>;
            ST(alloc_impl<T, M>(g));
            return geometry_impl<T, M>(g, xyz_host, mask_host, dval_host);
        });
    }
    if (s == WD_OK) s = count_active(g);
    if (s != WD_OK) {
        std::string keep = g_err;
        release(g);
        g_err = keep;
        return s;
    }
    *out = g;
    return WD_OK;
}

void wd_destroy_grid(wd_grid g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    release(g);
}

wd_status wd_set_stream(wd_grid g, void* cuda_stream)
{
    if (!g) return set_error(WD_ERR_INVALID_ARG, "grid is NULL");
    g->user_stream = (cudaStream_t)cuda_stream;
    return WD_OK;
}

static wd_status check_params(const wd_solve_params* p)
{
    if (!p) return set_error(WD_ERR_INVALID_ARG, "params is NULL");
    if (p->equation < 0 || p->equation > 2) return set_error(WD_ERR_INVALID_ARG, "bad equation");
    if (!(std::fabs(p->alpha_f) < 0.5)) return set_error(WD_ERR_INVALID_ARG, "|alpha_f| must be < 0.5");
    if (!(p->cfl > 0.0)) return set_error(WD_ERR_INVALID_ARG, "cfl must be positive");
    if (p->max_iters < 0 || p->poisson_max_iters < 0) return set_error(WD_ERR_INVALID_ARG, "negative iteration count");
    if (p->init < 0 || p->init > 2) return set_error(WD_ERR_INVALID_ARG, "bad init");
    return WD_OK;
}

wd_status wd_solve(wd_grid g, const wd_solve_params* p, void* phi_dev, wd_stats* stats)
{
    if (!g || !phi_dev) return set_error(WD_ERR_INVALID_ARG, "NULL grid or phi");
    ST(check_params(p));
    StreamGuard sg(g);
    auto t0 = std::chrono::steady_clock::now();
    wd_status s = dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        Solver<T, M> S(g, p);
        return S.solve(phi_dev, stats, false);
    });
    if (stats)
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return s;
}

wd_status wd_step_unsteady(wd_grid g, const uint8_t* mask_dev, const void* dval_dev,
                           const wd_solve_params* p, void* phi_dev, wd_stats* stats)
{
    if (!g || !phi_dev) return set_error(WD_ERR_INVALID_ARG, "NULL grid or phi");
    ST(check_params(p));
    StreamGuard sg(g);
    auto t0 = std::chrono::steady_clock::now();
    wd_status s = dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        if (mask_dev) ST(update_dirichlet(g, mask_dev, dval_dev));
        Solver<T, M> S(g, p);
        return S.solve(phi_dev, stats, true);
    });
    if (stats)
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return s;
}

// The solves of wd_solve, run as resumable tasks (Solver::begin .. finish) on the grids' own
// streams: every round queues one slice (check_every pseudo steps, a CUDA graph, and the copy
// of its change norms) of each unfinished solve before waiting for any, so the slices of all
// grids, whatever their shapes, run side by side on the GPU; each grid then gets exactly what
// wd_solve gives it alone (the same kernels, slices and convergence checks).
wd_status wd_solve_batch(wd_grid* grids, int n, const wd_solve_params* p, void** phi_dev,
                         wd_stats* stats)
{
    if (n < 0 || (n > 0 && (!grids || !phi_dev))) return set_error(WD_ERR_INVALID_ARG, "bad batch");
    ST(check_params(p));
    for (int i = 0; i < n; i++) {
        if (!grids[i] || !phi_dev[i]) return set_error(WD_ERR_INVALID_ARG, "NULL grid or phi in the batch");
        for (int k = 0; k < i; k++)
            if (grids[k] == grids[i]) return set_error(WD_ERR_INVALID_ARG, "a grid appears twice in the batch");
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<std::unique_ptr<StreamGuard>> guards;
    std::vector<std::unique_ptr<SolveTask>> tasks;
    std::vector<wd_status> rc(n, WD_OK);
    for (int i = 0; i < n; i++) {
        guards.emplace_back(new StreamGuard(grids[i]));
        tasks.emplace_back(make_solve_task(grids[i], p));
        rc[i] = tasks[i]->begin(phi_dev[i], false);
    }
    auto live = [&](int i) { return rc[i] == WD_OK && !tasks[i]->finished(); };
    for (;;) {
        bool any = false;
        for (int i = 0; i < n; i++)
            if (live(i)) {
                any = true;
                rc[i] = tasks[i]->enqueue();
            }
        if (!any) break;
        for (int i = 0; i < n; i++) {
            if (rc[i] != WD_OK || tasks[i]->finished()) continue;
            if (tasks[i]->check()) {
                const cudaError_t e = cudaStreamSynchronize(grid_stream(grids[i]));
                if (e != cudaSuccess) rc[i] = cuda_error(e, "wd_solve_batch");
            }
            if (rc[i] == WD_OK) rc[i] = tasks[i]->complete();
        }
    }
    wd_stats dummy;
    for (int i = 0; i < n; i++) {
        if (rc[i] == WD_OK || rc[i] == WD_ERR_NOT_CONVERGED || rc[i] == WD_ERR_DIVERGED)
            rc[i] = tasks[i]->finish(phi_dev[i], stats ? stats + i : &dummy);
    }
    wd_status first = WD_OK;
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < n; i++) {
        const cudaError_t e = cudaStreamSynchronize(grid_stream(grids[i]));
        if (e != cudaSuccess && rc[i] == WD_OK) rc[i] = cuda_error(e, "wd_solve_batch");
        if (stats) stats[i].seconds = sec;
        if (rc[i] != WD_OK && first == WD_OK) first = rc[i];
    }
    return first;
}

size_t wd_query_footprint(const wd_grid_desc* desc, const wd_solve_params* p)
{
    (void)p;
    if (validate_desc(desc) != WD_OK) return 0;
    return footprint_bytes(desc);
}

const char* wd_status_string(wd_status s)
{
    switch (s) {
    case WD_OK: return "ok";
    case WD_ERR_INVALID_ARG: return "invalid argument";
    case WD_ERR_OOM: return "out of device memory";
    case WD_ERR_CUDA: return "CUDA error";
    case WD_ERR_NOT_CONVERGED: return "not converged";
    case WD_ERR_DIVERGED: return "diverged";
    case WD_ERR_TIMEOUT: return "timeout";
    default: return "unknown status";
    }
}

const char* wd_last_error(void) { return g_err.c_str(); }

wd_status wd_get_metrics(wd_grid g, double* xi_dev, double* J_dev, double* dx_dev)
{
    if (!g) return set_error(WD_ERR_INVALID_ARG, "grid is NULL");
    StreamGuard sg(g);
    long long tot = g->D.total;
    size_t N = (size_t)g->D.n[0] * g->D.n[1] * g->D.n[2];
    for (int k = 0; k < 9 && xi_dev; k++) CK(from_padded(g, xi_dev + k * N, g->xi_d + k * tot, 8));
    if (J_dev) CK(from_padded(g, J_dev, g->J_d, 8));
    for (int k = 0; k < 3 && dx_dev; k++) CK(from_padded(g, dx_dev + k * N, g->dx_d + k * tot, 8));
    return WD_OK;
}

wd_status wd_derivative(wd_grid g, int dir, const void* in_dev, void* out_dev)
{
    if (!g || !in_dev || !out_dev || dir < 0 || dir >= g->desc.ndim)
        return set_error(WD_ERR_INVALID_ARG, "bad derivative arguments");
    StreamGuard sg(g);
    return dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        Solver<T, M> S(g, nullptr);
        CK(to_padded(g, g->w[W_T0], in_dev, sizeof(T)));
        ST(S.deriv_dir(dir, (const T*)g->w[W_T0], (T*)g->w[W_T1]));
        CK(from_padded(g, out_dev, g->w[W_T1], sizeof(T)));
        return WD_OK;
    });
}

wd_status wd_filter(wd_grid g, double alpha_f, int dir, const void* in_dev, void* out_dev)
{
    if (!g || !in_dev || !out_dev || dir < 0 || dir >= g->desc.ndim || !(std::fabs(alpha_f) < 0.5))
        return set_error(WD_ERR_INVALID_ARG, "bad filter arguments");
    StreamGuard sg(g);
    return dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        Solver<T, M> S(g, nullptr);
        CK(to_padded(g, g->w[W_T0], in_dev, sizeof(T)));
        ST(S.filter_dir(dir, alpha_f, (const T*)g->w[W_T0], (T*)g->w[W_T0]));
        CK(from_padded(g, out_dev, g->w[W_T0], sizeof(T)));
        return WD_OK;
    });
}

wd_status wd_rhs(wd_grid g, const wd_solve_params* p, int kind, const void* phi_dev, void* R_dev,
                 void* dt_dev)
{
    if (!g || !phi_dev || (kind != 0 && kind != 1)) return set_error(WD_ERR_INVALID_ARG, "bad rhs arguments");
    ST(check_params(p));
    StreamGuard sg(g);
    return dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        Solver<T, M> S(g, p);
        return S.rhs(kind, phi_dev, R_dev, dt_dev);
    });
}

wd_status wd_spalding(wd_grid g, const void* phip_dev, void* phi_dev)
{
    if (!g || !phip_dev || !phi_dev) return set_error(WD_ERR_INVALID_ARG, "bad spalding arguments");
    StreamGuard sg(g);
    return dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        Solver<T, M> S(g, nullptr);
        CK(to_padded(g, g->w[W_PHIN], phip_dev, sizeof(T)));
        ST(S.spalding_from_phin());
        CK(from_padded(g, phi_dev, g->w[W_PHIN], sizeof(T)));
        return WD_OK;
    });
}

wd_status wd_apply_bc(wd_grid g, void* phi_dev)
{
    if (!g || !phi_dev) return set_error(WD_ERR_INVALID_ARG, "bad bc arguments");
    StreamGuard sg(g);
    return dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        Solver<T, M> S(g, nullptr);
        CK(to_padded(g, g->w[W_PHIN], phi_dev, sizeof(T)));
        ST(S.bc((T*)g->w[W_PHIN], false));
        CK(from_padded(g, phi_dev, g->w[W_PHIN], sizeof(T)));
        return WD_OK;
    });
}

wd_status wd_steps(wd_grid g, const wd_solve_params* p, int kind, void* phi_dev, int nsteps,
                   wd_stats* stats)
{
    if (!g || !phi_dev || (kind != 0 && kind != 1) || nsteps < 0)
        return set_error(WD_ERR_INVALID_ARG, "bad steps arguments");
    ST(check_params(p));
    StreamGuard sg(g);
    return dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        Solver<T, M> S(g, p);
        return S.steps(kind, phi_dev, nsteps, stats);
    });
}

wd_status wd_reset_geometry(wd_grid g, const double* xyz_host, const uint8_t* mask_host,
                            const double* dval_host)
{
    if (!g || !xyz_host) return set_error(WD_ERR_INVALID_ARG, "NULL grid or xyz_host");
    wd_status s;
    {
        StreamGuard sg(g);
        s = dispatch(g, [&](auto* t, auto* m) {
            using T = std::remove_pointer_t<decltype(t)>;
            using M = std::remove_pointer_t<decltype(m)>;
            return geometry_impl<T, M>(g, xyz_host, mask_host, dval_host);
        });
    }
    if (s == WD_OK) s = count_active(g);
    return s;
}

wd_status wd_recede(wd_grid g, void* phi_dev, double s, double floor, uint8_t* mask_dev,
                    void* dval_dev)
{
    if (!g || !phi_dev || !mask_dev || !dval_dev) return set_error(WD_ERR_INVALID_ARG, "NULL argument");
    if (!(s >= 0.0) || !(floor <= 0.0)) return set_error(WD_ERR_INVALID_ARG, "need s >= 0 and floor <= 0");
    StreamGuard sg(g);
    const long long n = (long long)g->D.n[0] * g->D.n[1] * g->D.n[2];
    return dispatch(g, [&](auto* t, auto*) {
        using T = std::remove_pointer_t<decltype(t)>;
        CK(launch_recede<T>((T*)phi_dev, n, s, floor, mask_dev, (T*)dval_dev, g->stream));
        return WD_OK;
    });
}

wd_status wd_levelset(wd_grid g, void* phi_dev, double F, double dt, int nsteps)
{
    if (!g || !phi_dev || nsteps < 0 || !std::isfinite(F) || !(dt > 0.0) || !std::isfinite(dt))
        return set_error(WD_ERR_INVALID_ARG, "bad level-set arguments");
    StreamGuard sg(g);
    return dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        Solver<T, M> S(g, nullptr);
        return S.levelset(phi_dev, F, dt, nsteps);
    });
}

wd_status wd_level_length(wd_grid g, const void* phi_dev, double level, double* length)
{
    if (!g || !phi_dev || !length) return set_error(WD_ERR_INVALID_ARG, "NULL argument");
    if (g->D.ndim != 2 || g->batch != 1) return set_error(WD_ERR_INVALID_ARG, "single 2-D grids only");
    StreamGuard sg(g);
    const long long cells = (long long)(g->D.n[0] - !g->D.per[0]) * (g->D.n[1] - !g->D.per[1]);
    const int nb = (int)std::max<long long>(1, std::min<long long>((cells + 255) / 256, g->npartial));
    wd_status r = dispatch(g, [&](auto* t, auto*) {
        using T = std::remove_pointer_t<decltype(t)>;
        CK(launch_level_length<T>(g->D, (const T*)phi_dev, g->xyz, g->desc.period, level, g->partial,
                                  nb, g->stream));
        return WD_OK;
    });
    if (r != WD_OK) return r;
    std::vector<double> part(nb);
    CK(cudaMemcpyAsync(part.data(), g->partial, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    double sum = 0.0;
    for (int b = 0; b < nb; b++) sum += part[b];
    *length = sum;
    return WD_OK;
}

wd_status wd_get_tuning(wd_grid g, int* stage_threads, int* stencil_rows, int* batch_parts)
{
    if (!g) return set_error(WD_ERR_INVALID_ARG, "NULL grid");
    if (stage_threads) *stage_threads = g->tune_stage_threads;
    if (stencil_rows) *stencil_rows = g->tune_by;
    if (batch_parts) *batch_parts = g->tune_parts;
    return WD_OK;
}

wd_status wd_profile(wd_grid g, int enable)
{
    if (!g) return set_error(WD_ERR_INVALID_ARG, "grid is NULL");
    if (enable) {
        CK(prof_flush(g));
        for (int k = 0; k < WD_K_NCLASS; k++) {
            g->prof_ms[k] = 0.0;
            g->prof_n[k] = 0;
        }
    }
    g->prof_on = enable != 0;
    return WD_OK;
}

wd_status wd_profile_read(wd_grid g, int cls, double* ms_total, long long* launches)
{
    if (!g || cls < 0 || cls >= WD_K_NCLASS) return set_error(WD_ERR_INVALID_ARG, "bad profile query");
    CK(prof_flush(g));
    if (ms_total) *ms_total = g->prof_ms[cls];
    if (launches) *launches = g->prof_n[cls];
    return WD_OK;
}

}  // extern "C"

namespace wd {

template <typename T, typename M>
struct SolveTaskImpl final : SolveTask {
    wd_solve_params prm;      // the task's own copy; the solver points at it
    Solver<T, M> S;
    SolveTaskImpl(wd_grid g, const wd_solve_params* p) : prm(*p), S(g, &prm) {}
    wd_status begin(const void* phi, bool warm) override { return S.begin(phi, warm); }
    wd_status enqueue() override { return S.enqueue(); }
    wd_status complete() override { return S.complete(); }
    bool finished() const override { return S.finished(); }
    bool check() const override { return S.R.check; }
    wd_status finish(void* phi, wd_stats* st) override { return S.finish(phi, st); }
};

SolveTask* make_solve_task(wd_grid g, const wd_solve_params* p)
{
    SolveTask* out = nullptr;
    dispatch(g, [&](auto* t, auto* m) {
        using T = std::remove_pointer_t<decltype(t)>;
        using M = std::remove_pointer_t<decltype(m)>;
        out = new SolveTaskImpl<T, M>(g, p);
        return WD_OK;
    });
    return out;
}

cudaStream_t grid_stream(wd_grid g) { return g->stream; }
cudaStream_t grid_user_stream(wd_grid g) { return g->user_stream; }
size_t grid_bytes(wd_grid g) { return g->bytes; }
wd_status check_solve_params(const wd_solve_params* p) { return check_params(p); }

// merges a dense caller mask / Dirichlet values into the grid's Dirichlet set (walls kept)
// and recounts the active nodes; waits for the grid's stream
wd_status update_dirichlet(wd_grid g, const uint8_t* mask_dev, const void* dval_dev)
{
    wd_status s = dispatch(g, [&](auto* t, auto*) {
        using T = std::remove_pointer_t<decltype(t)>;
        CK(launch_mask_merge<T>(g->D, mask_dev, (const T*)dval_dev, g->mask, (T*)g->dval, g->wall,
                                g->stream));
        return WD_OK;
    });
    if (s != WD_OK) return s;
    return count_active(g);
}

}  // namespace wd
