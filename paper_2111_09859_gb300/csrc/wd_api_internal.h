// wd_api_internal.h -- host-side declarations shared by the libwd translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "wd.h"
#include "wd_internal.cuh"

namespace wd {

wd_status set_error(wd_status s, const char* msg);
wd_status cuda_error(cudaError_t e, const char* where);

bool dense_solve(int n, std::vector<double>& M, std::vector<double>& r);
bool filter_coefficients(int hw, double al, double* a);
void derivative_rows(int scheme, int N, int periodic, std::vector<double>& a,
                     std::vector<double>& c, int& implicit);
void filter_rows(double al, int N, int periodic, std::vector<double>& a, std::vector<double>& c,
                 int& implicit);
wd_status build_line_table(int N, int periodic, const std::vector<double>& a,
                           const std::vector<double>& c, int implicit, HostLineTab& tab);
void free_line_table(HostLineTab& tab);

// arguments of the pointwise stage kernel (right-hand side + RK4 stage update)
template <typename T, typename M>
struct StageArgs {
    const T* src;        // phi at which R is evaluated
    T* dst;              // stage output (RK modes) or R (rhs-only mode)
    const T* phin;       // state at the start of the pseudo step
    T* acc;              // running sum of the RK4 weights times R
    T* dt;               // local pseudo time step
    const T* U[3];       // grad(phi), physical components
    const T* lap;        // div(U)
    const T* kap;        // div(n) (curvature only)
    const T* lad;        // smoothed C|LAD| (LAD only)
    const T* adv;        // upwind U.grad(phi) (baseline scheme only; else |U|^2 is used)
    const M* sig1;       // sum_l |grad xi_l|
    const M* sig2;       // sum_l |grad xi_l|^2
    double eps, cfl;
    int equation, curvature, poisson;
};

// stage codes for launch_stage: 0..3 = RK4 stages, -1 = right-hand side and dt only
template <typename T, typename M>
cudaError_t launch_line(const Dims& D, int dir, const HostLineTab& tab, const LineOp& op, int nf,
                        int epi, const Fields<T>& f, const M* xi, int nU, int accumulate,
                        cudaStream_t st);
template <typename T, typename M>
cudaError_t launch_grad(const Dims& D, const T* const* Dl, const M* xi, T* const* U,
                        T* const* nv, double eps0, cudaStream_t st);
template <typename T, typename M>
cudaError_t launch_lad_raw(const Dims& D, const T* phi, const M* lads, double C, T* out,
                           cudaStream_t st);
template <typename T, typename M>
cudaError_t launch_stage(const Dims& D, const StageArgs<T, M>& a, int stage, cudaStream_t st);
template <typename T, typename M>
cudaError_t launch_spalding(const Dims& D, const T* const* U, const T* phip, T* phi,
                            cudaStream_t st);
template <typename T>
cudaError_t launch_bc_face(const Dims& D, int dir, int kind_lo, int kind_hi, const double* rlo,
                           const double* rhi, T* phi, cudaStream_t st);
template <typename T>
cudaError_t launch_bc_faces2d(const Dims& D, const int* klo, const int* khi, const double* const* rlo,
                              const double* const* rhi, const uint8_t* mask, const T* dval, int poisson, T* phi,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_bc_mask(const Dims& D, const uint8_t* mask, const T* dval, T* phi,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_norms(const Dims& D, const T* newp, T* oldp, const uint8_t* mask,
                         double* partial, unsigned* counter, double* result, int nblocks,
                         cudaStream_t st);
template <typename T>
cudaError_t launch_fill(T* p, long long n, T v, cudaStream_t st);

// constant metrics of a uniform Cartesian grid (cart != 0): d(xi_l)/d(x_m) = delta_lm ih[l]
template <typename M>
struct UwCart {
    int cart;
    M ih[3];
};

// baseline upwind advection term (wd_upwind.cu)
template <typename T, typename M>
cudaError_t launch_uw_adv(const Dims& D, const T* phi, const M* xi, const UwCart<M>& cc, T* adv,
                          cudaStream_t st);

// one RK4 stage of the level-set equation (wd_upwind.cu)
template <typename T, typename M>
struct LsArgs {
    const T* src;        // phi at which the stage evaluates F |grad phi|
    T* dst;              // stage output (aliases neither src nor phin)
    const T* phin;       // phi at the start of the step
    T* acc;              // running sum of the RK4 weights times the right-hand side
    const M* xi;         // 9 metric arrays d(xi_l)/d(x_m) at (l*3+m)
    UwCart<M> cc;        // or the constant metrics of a uniform Cartesian grid
    double F, dt;        // normal speed, time step
};
template <typename T, typename M>
cudaError_t launch_ls_stage(const Dims& D, const LsArgs<T, M>& a, int stage, cudaStream_t st);

template <typename T>
cudaError_t launch_recede(T* phi, long long n, double s, double floor, uint8_t* mask, T* dval,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_level_length(const Dims& D, const T* phi, const double* xyz,
                                const double (*period)[3], double level, double* part, int nblocks,
                                cudaStream_t st);
template <typename S, typename DT>
cudaError_t launch_convert(const S* in, DT* out, long long n, cudaStream_t st);
cudaError_t launch_unwrap(const Dims& D, int dir, const double* x, double shift, double* out,
                          cudaStream_t st);
cudaError_t launch_add_const(const Dims& D, double* p, double c, cudaStream_t st);
template <typename M>
cudaError_t launch_metric_finish(const Dims& D, const double* A, double* xi_d, double* J,
                                 double* dx, M* xi_m, M* sig1, M* sig2, cudaStream_t st);
template <typename M>
cudaError_t launch_lad_scale(const Dims& D, const double* xi_d, const double* dx, double ex,
                             M* lads, cudaStream_t st);
cudaError_t launch_ff_ratio(const Dims& D, const double* xyz, double* ratio, long long fmax,
                            cudaStream_t st);
template <typename T>
cudaError_t launch_mask_merge(const Dims& D, const uint8_t* src_dense, const T* val_dense,
                              uint8_t* mask, T* dval, const uint8_t* wallmask, cudaStream_t st);
cudaError_t launch_count(const Dims& D, const uint8_t* mask, unsigned long long* out,
                         cudaStream_t st);

// ---- solve tasks for the request loop ------------------------------------------------
// One solve of wd_solve split into device slices (see Solver::begin .. finish).
struct SolveTask {
    virtual ~SolveTask() {}
    virtual wd_status begin(const void* phi, bool warm) = 0;
    virtual wd_status enqueue() = 0;        // queues one slice (and its norm copy)
    virtual wd_status complete() = 0;       // host step after the slice has run
    virtual bool finished() const = 0;
    virtual bool check() const = 0;         // the last slice ends at a convergence check
    virtual wd_status finish(void* phi, wd_stats* stats) = 0;   // queues the copy-out
};
SolveTask* make_solve_task(wd_grid g, const wd_solve_params* p);
cudaStream_t grid_stream(wd_grid g);
cudaStream_t grid_user_stream(wd_grid g);
size_t grid_bytes(wd_grid g);
wd_status check_solve_params(const wd_solve_params* p);
wd_status update_dirichlet(wd_grid g, const uint8_t* mask_dev, const void* dval_dev);

}  // namespace wd
