/*
 * libvlasov -- GB300 (sm_103a) hot path of the moment-fitting PFC Vlasov
 * solver of Allmann-Rahn, Lautenbach and Grauer, "An Energy Conserving Vlasov
 * Solver That Tolerates Coarse Velocity Space Resolutions" (arXiv:2109.06743).
 *
 * C ABI. Plain pointers and sizes only. The library never allocates device
 * memory: every buffer is owned by the caller (for example allocated with
 * PyTorch) and must stay alive until vlasov_free. All compute calls are
 * asynchronous on the given CUDA stream (NULL = legacy default stream) and
 * return after enqueueing their kernels.
 *
 * Error behaviour: argument errors return VL_EINVAL immediately (nothing is
 * enqueued) and vl_last_error() describes them; a failed kernel launch returns
 * VL_ECUDA. Numeric errors found on the device (fit targets, i.e. moments of
 * f or fluid state, that are not finite or have n < 0) set the context's
 * status word; the next compute call on the context then returns VL_ENUMERIC
 * without enqueueing anything and clears the word, and vl_sync_status()
 * synchronises the stream and returns it. Because the calls are asynchronous
 * the error is returned by the first call made after the kernel that found
 * it has run (at the latest by vl_sync_status). Empty cells (n = 0) are not
 * an error. Newton non-convergence is not fatal: the continuous Maxwellian of
 * the targets is used and counted (vl_read_stats()). The status word is 4
 * bytes of pinned host memory mapped into the device, allocated by
 * vlasov_init and freed by vlasov_free (the only allocation of the library).
 * The library must not be used across a cudaDeviceReset of a device it has
 * run on (contexts and pfc_advect_v_static's cached scratch address refer to
 * that device's context).
 *
 * Layouts (row-major, fastest index last):
 *   f_s        [ny][nx][nvz][nvy][nvx] of float (precision 32) or double (64);
 *              1D1V: [nx][nv]. Velocity cell centres v_a(i) = vmin_a + (i+1/2) dv_a.
 *   moments    [ny*nx][20] double: raw midpoint sums dv^3 sum_c v^alpha f_c for
 *              alpha = 1, x, y, z, xx, xy, xz, yy, yz, zz, xxx, xxy, xxz, xyy,
 *              xyz, xzz, yyy, yyz, yzz, zzz (1D1V: [nx][4] = 1, v, vv, vvv).
 *   fluid      [nspecies][ny*nx][10] double: n, n u_a, int v_a v_b f dv
 *              (= P/m) in the order xx, xy, xz, yy, yz, zz (1D1V: [..][3]).
 *   yee        [6][ny+1][nx] double: Ex(i+1/2,j), Ey(i,j+1/2), Ez(i,j),
 *              Bx(i,j+1/2), By(i+1/2,j), Bz(i+1/2,j+1/2); planes with a j+1/2
 *              position use rows 0..ny-1 (2D3V only).
 *   eb         [ny*nx][6] double: E and B at cell centres (written by
 *              maxwell_step, read by pfc_advect_v and fluid_step).
 *   theta      [ny*nx][10] double: n', u'_a, Theta'_ab (xx,xy,xz,yy,yz,zz) of a
 *              fitted ten-moment Maxwellian (1D1V: [..][3]).
 * Normalisation of the paper (Sec. 2.1): mu0 = k_B = 1, eps0 = 1/c^2;
 * electrostatic 1D1V runs (Sec. 3.1) use eps0 = 1 and a Poisson solve.
 */
#ifndef VLASOV_H
#define VLASOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* vl_stream_t; /* a cudaStream_t */
typedef struct vl_ctx vl_ctx;             /* opaque, library-owned host object */

typedef enum {
    VL_OK = 0,
    VL_EINVAL = 1,   /* invalid argument or descriptor                    */
    VL_ECUDA = 2,    /* a CUDA call or kernel launch failed               */
    VL_ENOCONV = 3,  /* (stats only) Newton fallback was used             */
    VL_ENUMERIC = 4, /* non-finite or negative fit targets found on the device
                        (returned by the next call or by vl_sync_status) */
    VL_ENOTSUP = 5   /* valid but unsupported shape (e.g. non-cubic block) */
} vl_status;

#define VL_MAX_SPECIES 4

/* Problem descriptor (copied by vlasov_init). */
typedef struct {
    int nvdim;                      /* 1 (1D1V) or 3 (2D3V)                       */
    int nx, ny;                     /* spatial cells (ny = 1 for 1D1V)            */
    double x0, dx, y0, dy;          /* spatial cell edges and widths              */
    int bc_y;                       /* 0 periodic in y, 1 conducting/reflecting walls */
    int nspecies;                   /* 1..VL_MAX_SPECIES                          */
    double q[VL_MAX_SPECIES];       /* charge                                     */
    double m[VL_MAX_SPECIES];       /* mass                                       */
    int nv[VL_MAX_SPECIES][3];      /* velocity cells per axis (cubic for 2D3V)   */
    double vmin[VL_MAX_SPECIES][3]; /* velocity box, lower edge                   */
    double vmax[VL_MAX_SPECIES][3]; /* velocity box, upper edge                   */
    int precision;                  /* 32 or 64: element type of f                */
    int nshear;                     /* 5: exact Boris factorisation, 3: plain split */
    double c;                       /* speed of light (2D3V)                      */
    double ion_background;          /* fixed neutralising density (1D1V)          */
    double fit_tol;                 /* Newton tolerance relative to n (e.g. 1e-11) */
    int fit_max_iter;               /* Newton iteration cap (e.g. 20)             */
} vl_desc;

/* Bytes of caller-provided device workspace that vlasov_init needs for this
 * descriptor (shear tables, Newton parameters, fluid RK stages, counters).
 * Returns 0 for an invalid descriptor. */
size_t vlasov_work_bytes(const vl_desc* desc);

/* Create a context. f_dev[s] is species s's distribution function (layout
 * above, precision per desc), fluid_dev the fluid state, yee_dev the Yee
 * fields (2D3V; may be NULL for 1D1V), eb_dev the cell-centred fields,
 * work_dev/work_bytes the workspace (at least vlasov_work_bytes(desc), 256-byte
 * aligned). All pointers are device pointers owned by the caller. Validates
 * the descriptor (Sec. 3.3 walls need a velocity box symmetric in v_y).
 * f_dev, or any entry of it, may be NULL for a context that only runs the
 * fluid and field calls (the stand-alone fluid model): the calls that need
 * f then return VL_EINVAL. */
vl_status vlasov_init(const vl_desc* desc, void* const* f_dev, double* fluid_dev,
                      double* yee_dev, double* eb_dev, void* work_dev,
                      size_t work_bytes, vl_ctx** out);
vl_status vlasov_free(vl_ctx* ctx);
/* Human-readable description of the last error on this context (never NULL).
 * With ctx = NULL: the last error of a call made without a context (or that
 * failed before creating one) on the calling host thread. */
const char* vl_last_error(const vl_ctx* ctx);

/* Waits for the stream, then returns the context's status word: VL_ENUMERIC
 * if a kernel found non-finite or negative fit targets since the word was
 * last reported (the word is then cleared), VL_ECUDA if the stream failed,
 * else VL_OK. Paper Sec. 2.2 (the fit targets of Algorithm 1). */
vl_status vl_sync_status(vl_ctx* ctx, vl_stream_t stream);

/* Spatial PFC sweep of species s along axis 0 (x, periodic) or 1 (y, periodic
 * or reflecting walls with f(-y, v_y) = f(y, -v_y)), displacement v_a dt per
 * velocity cell, in place. Paper Sec. 2.1 (PFC scheme of Filbet et al. 2001)
 * and Sec. 3.3 (reflecting walls). |v| dt / dx may exceed 1. */
vl_status pfc_advect_x(vl_ctx* ctx, int species, int axis, double dt, vl_stream_t stream);

/* Spatial PFC sweeps of species s along x and then along y (the two
 * pfc_advect_x calls of the Vlasov step, Sec. 2.1 directional splitting;
 * Sec. 3.3 walls), fused into one pass that reads f once and writes it once.
 * Out of place: reads the species' current f and writes the result to f_out
 * (same layout, size and precision; caller-owned device memory that must not
 * overlap it and is aligned to the element size). On success the context's f
 * for species s becomes f_out, and the previous buffer is no longer used by
 * the context (the caller may pass it as f_out of the next call). The result
 * is element for element that of pfc_advect_x(x) then pfc_advect_x(y); the
 * same limits apply (VL_EINVAL). Grids whose nx or ny is not a multiple of 8,
 * or whose y shift exceeds 6 cells, take the two single-axis sweeps in place
 * followed by a device copy into f_out, with the same result. */
vl_status pfc_advect_xy(vl_ctx* ctx, int species, double dt, void* f_out, vl_stream_t stream);

/* Velocity-space PFC advection of species s under (q/m)(E + v x B) over dt
 * with the cell-centred fields eb, zero-flux at the velocity box (Sec. 2.1).
 * 2D3V: the Boris map of each cell is factored into nshear single-axis
 * shears, all applied to the block in shared memory. If mom_out is not NULL
 * the raw moments of the advected f are written there ([ncell][20], fused
 * epilogue, Sec. 2.1 moments). In place. */
vl_status pfc_advect_v(vl_ctx* ctx, int species, double dt, double* mom_out,
                       vl_stream_t stream);

/* pfc_advect_v without a context or workspace: the same velocity pass for
 * `ncell` consecutive cells given by plain device pointers, with its per-cell
 * scratch (20 doubles per cell: the shear factors of the velocity map) in a
 * fixed static device array of the library instead of a caller workspace.
 * It allocates no memory, host or device. The paper has no counterpart: it
 * serves callers that may not allocate device memory (hosts that own every
 * device byte through an arena fixed before the run; latency-bound callers
 * for which an allocation or its failure mid-step is not acceptable).
 *   desc      validated like vlasov_init's; species s selects q, m and the box
 *   f_dev     [ncell][V] species-s velocity blocks in desc->precision, in place
 *   eb_dev    [ncell][6] double, cell-centred E and B of those cells
 *   mom_out   [ncell][20] raw moments of the result, or NULL
 * At most VL_STATIC_SCRATCH_CELLS cells per call (VL_EINVAL beyond that:
 * split the call by cell ranges); ncell == 0 does nothing. The first call on
 * each device resolves the array's address (a runtime query, not a stream
 * operation) with that device current; make it before any stream capture.
 * Every call shares the array: nothing in it has to start at zero (each call
 * writes every row it reads), but calls that overlap in time on one device
 * race on it. f_dev must be aligned to its element size, eb_dev and mom_out
 * to 8 bytes, and mom_out must not overlap f_dev (VL_EINVAL otherwise,
 * before any launch). The cached address is that of the device's current
 * context: do not call across a cudaDeviceReset. Errors are reported through
 * vl_last_error(NULL) on the calling thread. */
#define VL_STATIC_SCRATCH_CELLS 32768
vl_status pfc_advect_v_static(const vl_desc* desc, int species, void* f_dev,
                              const double* eb_dev, long long ncell, double dt,
                              double* mom_out, vl_stream_t stream);

/* Raw midpoint moments of species s (Sec. 2.1), [ncell][20] (1D1V: [ncell][4]). */
vl_status moments(vl_ctx* ctx, int species, double* mom_out, vl_stream_t stream);

/* Moment fitting of Algorithm 1 (Sec. 2.2) for species s. vmom: raw moments
 * of the current f ([ncell][20], e.g. from pfc_advect_v). The fluid moments
 * of the context are rescaled by n_V/n_F; two discrete Maxwellians are fitted
 * by Newton iteration (their midpoint moments of degree <= 2 equal the
 * V and the rescaled F targets; precision 64: plain FP64 arithmetic;
 * precision 32: double-float arithmetic, about 44 significant bits, on the
 * FP32 pipe, with an FP32 Jacobian); then f <- f - f_M,V + f_M,F, negative values
 * are clipped and the cell rescaled to n_V (limiter of Algorithm 1). The
 * fluid state is replaced by its rescaled moments. use_mlp != 0 starts Newton
 * from the network's prediction (see the MLP section below; needs weights
 * from mlp_init/mlp_train or mlp_set_weights) instead of the continuous
 * Maxwellian, with the cold start as the fallback. If theta_v/theta_f are not NULL the fitted parameters are
 * written there. If mom_out is not NULL the raw moments of the new f are
 * written there. In place on f and the fluid state. */
vl_status moment_fit(vl_ctx* ctx, int species, const double* vmom, int use_mlp,
                     double* theta_v, double* theta_f, double* mom_out,
                     vl_stream_t stream);

/* The two halves of moment_fit, for callers that schedule or time them
 * separately: moment_fit_solve runs the Newton fits, keeps their
 * coefficients in the context's workspace (and writes theta_v/theta_f if not
 * NULL) and rescales the fluid state; moment_fit_exchange then applies
 * f <- f - f_M,V + f_M,F and the limiter with the Maxwellians of the
 * preceding solve of the same species. */
vl_status moment_fit_solve(vl_ctx* ctx, int species, const double* vmom, int use_mlp,
                           double* theta_v, double* theta_f, vl_stream_t stream);
vl_status moment_fit_exchange(vl_ctx* ctx, int species, const double* vmom,
                              double* mom_out, vl_stream_t stream);

/* Selects how the double-float 2D3V Newton fits of this species (precision
 * 32; Sec. 2.2, Algorithm 1's moment fitting) evaluate a discrete Maxwellian
 * whose values span more than the float range over the velocity block, i.e.
 * one that is narrow against a velocity box sized for a hotter population
 * (values falling below e^-80 of the peak towards the box's corners).
 * wide < 0 (the default): chosen on the device at every fit from the targets,
 * without a host synchronisation: the wide kernel if some cell with at least
 * 1e-10 of the largest density has a V or F Maxwellian that falls by more
 * than 60 e-folds from its peak to the farthest corner of the box, else the
 * common one (both kernels are launched; the one not chosen returns at
 * once). wide = 0: always the common kernel (one FP64 exponential per
 * velocity cell for such blocks). wide = 1: always the kernel that also
 * holds the centre-out double-float recurrences, which evaluate such blocks
 * at the common evaluation's speed. The fitted Maxwellians agree to rounding
 * either way; vl_read_stats counts the fits of the wide kernel. Takes effect
 * from the next moment_fit(_solve) of the species; host only, no launch.
 * VL_EINVAL for a bad species. */
vl_status moment_fit_wide(vl_ctx* ctx, int species, int wide);

/* One SSP-RK3 step (Shu-Osher 1988) of the ten-moment equations of Sec. 2.1
 * for every species with CWENO fluxes (Kurganov-Levy 2000). The third moments
 * come from mom_t[s] (stage 1), mom_t1[s] (stage 2) and their average
 * (stage 3), both raw moment arrays [ncell][20] (1D1V: [ncell][4]); E and B
 * are the cell-centred fields of the context, frozen over the step. */
vl_status fluid_step(vl_ctx* ctx, double dt, const double* const* mom_t,
                     const double* const* mom_t1, vl_stream_t stream);

/* fluid_step for species s alone (its raw moments mom_t, mom_t1). Each
 * species' fluid state evolves with its own moments and the frozen fields,
 * so the species may be stepped separately, in any order: a caller can run
 * one species' fluid step, fit and exchange before the next species' sweeps
 * (and start moving its f while the next species computes). Uses the
 * workspace's fluid stage buffers, so calls for different species on
 * different streams must not overlap. */
vl_status fluid_step_species(vl_ctx* ctx, int species, double dt, const double* mom_t,
                             const double* mom_t1, vl_stream_t stream);

/* The stand-alone ten-moment fluid model with the gradient heat-flux closure
 * (Sec. 2.3, Eq. "gradient closure"): one SSP-RK3 step of length dt of every
 * species' fluid state, E and B frozen at the context's cell-centred fields.
 * The third moment in the flux is that of the Maxwellian with the state's
 * n, u and E2 (zero heat flux), and the heat flux enters as
 * -(1/m) div Q = (chi / k_s0) n v_t lap(theta) in the second-moment equation,
 * theta = E2/n - u u, v_t = sqrt(tr(theta)/3), chi = 2 sqrt(2/pi) and
 * k_s0 = 1/d_s with d_s = sqrt(m_s/(n0 q_s^2)) at the reference density
 * n0 = 1 (mu0 = 1). No kinetic moments are used; with maxwell_step(h, NULL)
 * for the fields (current of the fluid state) it is the paper's fluid solver.
 * 2D3V only (VL_EINVAL otherwise); uses the workspace's fluid stage buffers. */
vl_status fluid_step_closure(vl_ctx* ctx, double dt, vl_stream_t stream);

/* Field update. 2D3V: one leapfrog Yee step of length h (B h/2, E h, B h/2)
 * with the current sum_s q_s n_s u_s taken from mom[s] (raw moments) or, if
 * mom is NULL, from the fluid state; then the cell-centred eb. 1D1V: Poisson
 * solve dE/dx = rho with rho = ion_background + sum_s q_s n_s (h unused).
 * Paper Sec. 2.1 (FDTD, two half steps per time step) and Sec. 3.1. */
vl_status maxwell_step(vl_ctx* ctx, double h, const double* const* mom,
                       vl_stream_t stream);

/* ---- MLP warm start of the moment fit (Sec. 2.2; the learned part) --------
 * A 12 -> 128 -> 128 -> 10 GELU network predicts, per fit, the Newton
 * solution minus the cold start (eta* - eta_0 in the fit's scaled
 * coordinates) from 12 inputs of the fit targets: Theta_ab/(dv_a dv_b) (6),
 * (u_a - nearest cell centre)/dv_a (3), (u_a - vmin_a)/(vmax_a - vmin_a) (3).
 * moment_fit_solve(use_mlp = 1) starts Newton there; Newton still runs to
 * fit_tol and restarts from the cold start if the warm run fails, so the
 * fitted Maxwellians do not depend on the network. All GEMMs (inference and
 * training) run on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation). The parameters live in the context's workspace as FP32:
 *   xm[12] xs[12] ym[10] ys[10] ysc[10] | W1[128][12] b1[128] | W2[128][128]
 *   b2[128] | W3[10][128] b3[10]  (W[out][in]; inputs standardised by xm,
 *   xs; the network's outputs are y = asinh(t / ysc) standardised by ym, ys).
 *   Training samples: VL_MLP_SAMPLE floats each, x[12], t[10]
 *   (= eta* - eta_0), flag (1 = usable), pad. */
#define VL_MLP_NPARAM 19520
#define VL_MLP_SAMPLE 24

/* Random (Glorot-uniform, seeded) weights, zero biases, unit normalisation,
 * cleared Adam state. Synchronous. */
vl_status mlp_init(vl_ctx* ctx, unsigned long long seed);
/* Copy VL_MLP_NPARAM floats from / to host memory. Synchronous. */
vl_status mlp_set_weights(vl_ctx* ctx, const float* w_host);
vl_status mlp_get_weights(vl_ctx* ctx, float* w_host);
/* From the next moment_fit_solve on, every converged 2D3V fit appends one
 * training sample to samples_dev (device, capacity samples; later fits are
 * dropped); capacity 0 stops harvesting. Resets the count. */
vl_status mlp_set_harvest(vl_ctx* ctx, float* samples_dev, long long capacity, vl_stream_t stream);
/* Number of samples harvested so far (at most the capacity). Synchronises. */
vl_status mlp_harvest_count(vl_ctx* ctx, long long* n, vl_stream_t stream);
/* Normalisation constants from n samples: input means and deviations;
 * output scales ysc = geometric means of |t| (at least 1e-6), then the means
 * ym of asinh(t / ysc) and ys = max(1, their deviations). */
vl_status mlp_normalize(vl_ctx* ctx, const float* samples_dev, long long n, vl_stream_t stream);
/* `steps` Adam steps (lr, beta 0.9 / 0.999) on the mean-square error of the
 * standardised transformed outputs, each on `batch` samples (a multiple of 128) drawn
 * from the n samples by a counter hash of seed and the step. loss_host (or
 * NULL) receives the loss of every step (synchronises per step). */
vl_status mlp_train(vl_ctx* ctx, const float* samples_dev, long long n, int steps, int batch,
                    float lr, unsigned long long seed, double* loss_host, vl_stream_t stream);
/* The network on raw inputs x_dev[n][12] -> y_dev[n][10] (eta* - eta_0);
 * NaN rows of inputs give NaN outputs. Synchronises. */
vl_status mlp_forward(vl_ctx* ctx, const float* x_dev, long long n, float* y_dev, vl_stream_t stream);
/* Gradient of the training loss (mean over the n samples and 10 outputs of
 * the squared error of the standardised transformed outputs) with respect to all VL_MLP_NPARAM
 * parameters (zero for the normalisation constants) into grad_dev, and the
 * loss into *loss_host (or NULL). Synchronises. */
vl_status mlp_grad(vl_ctx* ctx, const float* samples_dev, long long n, float* grad_dev,
                   double* loss_host, vl_stream_t stream);

/* Device counters accumulated since the last reset: out[0] Newton
 * iterations, out[1] Newton fallbacks, out[2] clipped cells, out[3] fits
 * whose targets are invalid (empty, non-finite or not positive definite);
 * the work of the double-float 2D3V Newton fits (precision 32; each counted
 * once per fit and evaluation, over the whole velocity block): out[4]
 * double-float moment evaluations (recurrence path), out[5] FP32 Jacobian
 * (Gram) evaluations, out[6] evaluations with one FP64 exponential per
 * velocity cell (wide exponent range), out[7] Newton steps with the FP64
 * Jacobian; out[8] asynchronous tile copies whose wait ran out of time (the
 * fused spatial sweep gives up on such a tile and leaves it unwritten: any
 * nonzero value means the result of that call is invalid); out[9] fits run
 * by the wide double-float kernel; the work of the FP64 fits (precision 64):
 * out[10] moment evaluations, out[11] of which with the Gram sums; out[12]
 * fits started from the network's prediction (use_mlp, prediction accepted
 * by the network's input and output range guard). Synchronises the stream. */
#define VL_NSTATS 13
vl_status vl_read_stats(vl_ctx* ctx, long long out[VL_NSTATS], vl_stream_t stream);
vl_status vl_reset_stats(vl_ctx* ctx, vl_stream_t stream);

/* Number of kernels this library has launched (all contexts, process-wide). */
long long vl_launch_count(void);

/* Measured fused multiply-add throughput of the current device in FP32
 * (precision 32) or FP64 (64), in operations per second (a fused
 * multiply-add counted as one operation): a kernel of independent FMA
 * chains, eight 256-thread blocks per SM, timed with CUDA events on the
 * stream after one untimed launch; it changes no device setting. The
 * denominator of the Newton fits' ALU roofline; the paper has no
 * counterpart. sink_dev: 8 bytes of device memory (8-byte aligned) that the
 * kernel could write but never does. Synchronises the stream. */
vl_status vl_fma_peak(int precision, double* ops_per_s, void* sink_dev, vl_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif
