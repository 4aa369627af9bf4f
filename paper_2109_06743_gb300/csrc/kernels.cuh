// Kernel argument structs and host-side launchers of libvlasov.
#pragma once

#include "common.cuh"

namespace vl {

// ---- spatial PFC sweep ----------------------------------------------------
struct SpaceSweepArgs {
    void* f;
    int n;                  // cells along the sweep axis
    long long row_stride;   // elements between neighbouring cells along the line
    long long line_stride;  // elements between neighbouring lines
    int nlines;             // number of lines
    long long V;            // velocity block size
    int wall;               // reflecting walls (mirror rows use the v_y-mirrored column)
    int ncol, nchunks;      // velocity columns per tile, tiles per line
    int mode;               // 0: contiguous columns, 1: v_y mirror pairs, 2: two v_y rows + mirrors
    int vec;                // column runs 16-byte aligned: stage tiles with cp.async
    int nbuf;               // tile buffers in shared memory (2: prefetch the next tile)
    int nvx, nvy;
    int axis_div, axis_mod; // velocity index of the sweep axis: (vi / div) % mod
    double vmin_a, dv_a, dt_over_h;
};
cudaError_t launch_pfc_space(const SpaceSweepArgs& a, int precision, cudaStream_t st);

// ---- fused x + y spatial sweep (out of place) ------------------------------
// Division of 0 <= n < 2^31 by a fixed d >= 1 with a multiply-high (the
// round-up method of Granlund and Montgomery, 1994): q = (hi(n m) + n) >> l,
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1 (mod 2^32).
struct FastDiv {
    unsigned m;
    int l;
    int d;
};
inline FastDiv make_fastdiv(int d) {
    FastDiv f;
    int l = 0;
    while ((1LL << l) < d) ++l;
    f.l = l;
    f.m = (unsigned)((((1ULL << 32) * ((1ULL << l) - (unsigned long long)d)) / (unsigned long long)d) + 1ULL);
    f.d = d;
    return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
    return (int)(((unsigned long long)__umulhi((unsigned)n, f.m) + (unsigned)n) >> f.l);
}
#endif
struct SpaceXYArgs {
    const void* f_in;       // [ny][nx][V], read only
    void* f_out;            // [ny][nx][V], must not overlap f_in
    int nx, ny;
    long long V;            // velocity block size
    int nvx, nvy;
    int wall;               // reflecting walls in y (mirror rows use the v_y-mirrored column)
    int ncol, nchunks;      // contiguous velocity columns per tile, ceil(V / ncol)
    int tx, ty;             // spatial tile; tx | nx, ty | ny, both multiples of 8
    int hx;                 // halo cells on each side in x: largest x shift + 2
    int hy;                 // halo rows on each side: largest y shift + 2 (<= ny)
    unsigned long long* counters;  // device counters (lost tile copies)
    FastDiv div_nvx, div_nvy;      // filled by the launcher
    FastDiv div_ntx, div_tpc;      // tiles along x, tiles per velocity chunk (TMA path)
    FastDiv div_bx;                // cells per input box row (TMA path)
    double vminx, dvx, cx;  // v_x box and dt / dx
    double vminy, dvy, cy;  // v_y box and dt / dy
};
size_t pfc_space_xy_smem(const SpaceXYArgs& a, int precision);
cudaError_t launch_pfc_space_xy(const SpaceXYArgs& a, int precision, cudaStream_t st);

// ---- velocity-space PFC pass (+ fused moments) -----------------------------
// Centred-index moments -> physical raw moments: out[o] = sum_t coef[o][t] *
// im[idx[o][t]], t < nterm[o] (binomial expansion of v = vc + dv xi, times dv^3).
struct MomConv {
    double coef[20][8];
    unsigned char idx[20][8];
    unsigned char nterm[20];
};
void make_mom_conv(const double* vmin, const double* dv, int n, MomConv* out);

struct VelocityArgs {
    void* f;
    const double* eb;       // [ncell][6]
    double* shears;         // [ncell][5][4] workspace
    double* mom_out;        // [ncell][20] or null
    long long ncell;
    int nv;                 // cubic block edge (2D3V); 1D1V: line length
    int nshear;
    int nbuf;               // block buffers in shared memory (set by the launcher)
    int vec;                // f is 16-byte aligned: write blocks back with 16-byte stores (set by the launcher)
    double qm, dt;
    double vmin[3], dv[3];
    MomConv conv;
};
cudaError_t launch_velocity(const VelocityArgs& a, int nvdim, int precision, cudaStream_t st);
// address of the static scratch of pfc_advect_v_static on the current device
cudaError_t static_scratch_address(void** out);

struct MomentArgs {
    const void* f;
    double* mom_out;
    long long ncell;
    int nv;
    double vmin[3], dv[3];
    MomConv conv;
};
cudaError_t launch_moments(const MomentArgs& a, int nvdim, int precision, cudaStream_t st);

// ---- moment fitting ----------------------------------------------------------
struct FitArgs {
    const double* vmom;     // [ncell][nmom] raw moments of f
    double* fluid;          // [ncell][ncomp] fluid state (rescaled in place)
    double* coef_v;         // [ncell][16] fit coefficients (eta, u0, sigma) of f_M,V
    double* coef_f;         // [ncell][16] of f_M,F
    int* status;            // [ncell][2]
    unsigned long long* counters;
    const float* warm;      // [ncell][2][10] predicted eta* - eta_0 (MLP), or null: cold start
    float* harvest;         // training samples of converged fits, or null
    long long harvest_cap;
    unsigned long long* harvest_count;
    long long ncell;
    int nv;
    double vmin[3], dv[3], vmax[3];
    double tol;
    int max_iter;
    int wide;               // 1: the fit kernel with the centre-out evaluation, 0: the common
                            // one, -1: chosen on the device from select (moment_fit_wide)
    const unsigned long long* select;  // wide = -1: [2] FP64 bits of the largest n over all
                            // cells and over the cells that need the wide kernel (fit_select)
    int fp64;               // 1: the plain FP64 fit (FP64 mode), 0: double-float on the FP32 pipe
    int* numeric;           // status word (device-visible host memory): set to VL_ENUMERIC when
                            // a target is not finite or has n < 0; may be null
};
cudaError_t launch_fit(const FitArgs& a, int nvdim, cudaStream_t st);
// auto choice of the 2D3V fit kernel: sel[0], sel[1] (zeroed by the caller) get
// the FP64 bits of the largest n over all cells and over the cells whose V or
// F Maxwellian falls by more than 60 e-folds from its peak to the farthest
// corner of the velocity box
cudaError_t launch_fit_select(const FitArgs& a, unsigned long long* sel, cudaStream_t st);

// ---- MLP warm start (mlp.cu) ------------------------------------------------------
struct MlpInferArgs {
    const float* w;         // parameter blob (FP32)
    int mode;               // 0: inputs from fit targets; 1: raw inputs x
    const double* vmom;     // mode 0: [ncell][nmom] moments of f
    const double* fluid;    // mode 0: [ncell][10] fluid state (not modified)
    int nmom;
    const float* x;         // mode 1: [nfit][12]
    long long nfit;         // mode 0: 2 * ncell (fit 2c: V, 2c + 1: F)
    double vmin[3], dv[3], vmax[3];
    float* y;               // [nfit][10] eta* - eta_0 (NaN: no usable input)
    int* err;               // set to 1 if a tensor-core wait timed out
};
struct MlpTrainArgs {
    const float* w;
    float* grad;            // [NPARAM] accumulated
    double* loss;           // accumulated sum of squares
    const float* samples;
    long long n;
    int mode;               // 0: rows drawn by a counter hash of (seed, row); 1: rows row0 + r
    long long rows, row0;
    unsigned long long seed;
    float inv_count;        // 1 / (rows * 10)
    int* err;
};
cudaError_t launch_mlp_stats(const float* samples, long long n, double* acc, float* w, cudaStream_t st);
cudaError_t launch_mlp_infer(const MlpInferArgs& a, cudaStream_t st);
cudaError_t launch_mlp_train_step(const MlpTrainArgs& a, cudaStream_t st);
cudaError_t launch_mlp_adam(float* w, float* m, float* v, const float* g, float lr, int step, cudaStream_t st);
cudaError_t launch_newton3d(const FitArgs& a, cudaStream_t st);
cudaError_t launch_theta(const double* coef, const int* status, int which, double* theta, long long ncell, int nvdim,
                         cudaStream_t st);

struct ExchangeArgs {
    void* f;
    const double* vmom;     // [ncell][nmom] (n_V)
    const double* coef_v;
    const double* coef_f;
    const int* status;
    double* mom_out;        // moments of the new f or null
    unsigned long long* counters;
    double* par;            // [ncell][2][10] scratch: Maxwellian line parameters
    long long ncell;
    int nv;
    double vmin[3], dv[3];
    MomConv conv;
};
cudaError_t launch_exchange(const ExchangeArgs& a, int nvdim, int precision, cudaStream_t st);

// ---- fluid ---------------------------------------------------------------------
struct FluidArgs {
    double* U;              // [ncell][ncomp] state (updated by the last stage)
    const double* Us;       // stage input
    double* Uout;           // stage output
    const double* U0;       // state at t (for the RK combination)
    const double* q0;       // raw moments with the third moments at offset qoff
    const double* q1;
    double wq0, wq1;        // Q = wq0 * q0 + wq1 * q1
    const double* eb;
    int nx, ny, bc_y, nvdim, nmom;
    int precision;          // 64: right-hand side in FP64; 32: in FP32 (state FP64)
    double dx, dy, qm, dt;
    double a0, a1;          // Uout = a0 * U0 + a1 * (Us + dt L(Us))
    float* Usf;             // FP32 mode: [ncell][10] stage input converted once (or null)
    float* Qf;              // FP32 mode: [ncell][10] weighted third moments (or null)
    int closure;            // 1: gradient-closure model (third moment of the state's
                            // Maxwellian, heat flux as chi_k0 n v_t lap theta); q0, q1 unused
    double chi_k0;          // chi / k_s0 of the closure
};
cudaError_t launch_fluid_stage(const FluidArgs& a, cudaStream_t st);

// ---- fields --------------------------------------------------------------------
struct FieldArgs {
    double* yee;            // [6][ny+1][nx]
    double* eb;             // [ncell][6]
    const double* cur;      // [ncell][3]
    int nx, ny, wall;
    double dx, dy, c2, h;
};
cudaError_t launch_current(double* cur, const double* const* src, const double* q, int nspecies,
                           int stride, int off, long long ncell, int nvdim, double bg, cudaStream_t st);
cudaError_t launch_maxwell(const FieldArgs& a, cudaStream_t st);
cudaError_t launch_poisson(const double* rho, double* eb, int nx, double dx, cudaStream_t st);

// ---- measured FMA peak (probe.cu) ---------------------------------------------
cudaError_t fma_peak(int precision, double* ops_per_s, void* sink, cudaStream_t st);

}  // namespace vl
