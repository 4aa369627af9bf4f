// Shared device-side definitions of libvlasov (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vlasov.h"

namespace vl {

constexpr int kMaxSpecies = VL_MAX_SPECIES;

// Per-species constants passed by value to kernels.
struct SpeciesParams {
    double q, m, qm;
    int nv[3];
    double vmin[3], dv[3];
    long long vblock;  // cells per velocity block
};

// Grid constants passed by value to kernels.
struct GridParams {
    int nvdim, nx, ny, bc_y;
    double x0, dx, y0, dy;
    long long ncell;
};

// Process-wide launch counter (reported by vl_launch_count).
void count_launch(int n = 1);

// Workspace layout offsets (bytes) computed by the ABI layer.
struct Workspace {
    double* cellwork;     // [ncell][20] per-cell scratch: the shear factors of the velocity
                          // map (pfc_advect_v), then the Maxwellian line parameters of
                          // the exchange (moment_fit_exchange)
    double* coef_v;       // [ncell][16] fit coefficients of f_M,V
    double* coef_f;       // [ncell][16] fit coefficients of f_M,F
    int* fit_status;      // [ncell][2] status of the V and F fits
    double* fluid_u1;     // [ncell][10] RK stage 1 (per call, reused per species)
    double* fluid_u2;     // [ncell][10]
    double* fluid_l;      // [ncell][10]
    double* cur;          // [ncell][3] current density at cell centres
    float* fluid_f;       // [2][ncell][10] FP32 copies of a stage's state and third moments
    unsigned long long* counters;  // [VL_NSTATS]
    unsigned long long* fit_select;  // [2] device-side choice of the fit kernel (fit_select_kernel)
    float* mlp;           // MLP weights and scratch
};

// indices of the device counters (vl_read_stats)
enum { CNT_ITERS = 0, CNT_FALLBACK = 1, CNT_CLIPPED = 2, CNT_INVALID = 3, CNT_EVAL_M = 4, CNT_EVAL_G = 5,
       CNT_EVAL_SLOW = 6, CNT_PRECISE = 7, CNT_COPY_TIMEOUT = 8, CNT_WIDE_FITS = 9, CNT_EVAL64_M = 10,
       CNT_EVAL64_G = 11, CNT_WARM = 12 };

__host__ __device__ inline int ifloor(double x) { return (int)floor(x); }

}  // namespace vl
