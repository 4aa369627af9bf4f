// MLP warm start of the moment fit (see mlp_common.cuh): inference over all
// fits of a species, training steps (forward, loss, backward, gradient
// accumulation) and the Adam update. Every GEMM runs on the tensor cores
// through tcgen05 (tc.cuh): BF16 operands staged in shared memory, FP32
// accumulators in TMEM. A CTA of 128 threads handles 128 samples: thread t
// owns sample t, which is TMEM lane t of every [128 x N] product, so the
// epilogues (bias, GELU, its derivative, loss) read their row with
// tcgen05.ld and write the next operand straight back to shared memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "mlp_common.cuh"
#include "tc.cuh"

namespace vl {

using namespace mlp;

namespace {

constexpr int kT = 128;  // samples per tile = threads per CTA
constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ void put_bf16(unsigned char* base, int off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16(v);
}

// weights (FP32 blob) -> BF16 operands in shared memory, K-major:
// W1 [128 x 16] (K padded), W2 [128 x 128], W3 [16 x 128] (N padded), and for
// training the transposed W2T [128 x 128] and W3T [128 x 16]
__device__ void stage_weights(const float* w, unsigned char* sW1, unsigned char* sW2, unsigned char* sW3,
                              unsigned char* sW2T, unsigned char* sW3T) {
    for (int e = threadIdx.x; e < kHid * 16; e += blockDim.x) {
        const int o = e / 16, i = e % 16;
        put_bf16(sW1, tc::kmajor_offset(o, i, kHid), i < kIn ? w[kOffW1 + o * kIn + i] : 0.f);
    }
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
        const int o = e / kHid, i = e % kHid;
        const float v = w[kOffW2 + e];
        put_bf16(sW2, tc::kmajor_offset(o, i, kHid), v);
        if (sW2T) put_bf16(sW2T, tc::kmajor_offset(i, o, kHid), v);
    }
    for (int e = threadIdx.x; e < 16 * kHid; e += blockDim.x) {
        const int o = e / kHid, i = e % kHid;
        const float v = o < kOut ? w[kOffW3 + o * kHid + i] : 0.f;
        put_bf16(sW3, tc::kmajor_offset(o, i, 16), v);
        if (sW3T) put_bf16(sW3T, tc::kmajor_offset(i, o, kHid), v);
    }
}

struct TcState {
    uint64_t* bar;
    uint32_t phase;
    bool ok;
    // make shared-memory operands visible to the tensor core, then one thread
    // issues the queued products (the lambda) and commits; everyone waits
    template <typename Issue>
    __device__ __forceinline__ void run(Issue issue) {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x == 0) {
            issue();
            tc::mma_commit(bar);
        }
        ok = tc::mbar_wait(bar, phase & 1u) && ok;
        ++phase;
        tc::fence_after_sync();
    }
};

__device__ __forceinline__ void flag_error(int* err, bool ok) {
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace

// ------------------------------------------------------------------ statistics

// Statistics of the usable samples. Pass 0: sums and sums of squares of the
// inputs and sums of log |t_k| (acc[0..11], [12..23], [24..33]); pass 1:
// sums and sums of squares of y_k = asinh(t_k / s_k) (acc[34..43],
// [44..53]); acc[54] counts the samples.
__global__ void mlp_stats_kernel(const float* samples, long long n, const float* w, int pass, double* acc) {
    __shared__ double s[55];
    if (threadIdx.x < 55) s[threadIdx.x] = 0.0;
    __syncthreads();
    double loc[34];
    for (int q = 0; q < 34; ++q) loc[q] = 0.0;
    double cnt = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float* p = samples + i * kSample;
        if (p[22] != 1.f) continue;
        if (pass == 0) {
            for (int q = 0; q < kIn; ++q) {
                const double v = p[q];
                loc[q] += v;
                loc[kIn + q] += v * v;
            }
            for (int k = 0; k < kOut; ++k) loc[24 + k] += log(fabs((double)p[kIn + k]) + 1e-30);
        } else {
            for (int k = 0; k < kOut; ++k) {
                const double y = asinh((double)p[kIn + k] / (double)w[kOffYsc + k]);
                loc[k] += y;
                loc[kOut + k] += y * y;
            }
        }
        cnt += 1.0;
    }
    const int nq = pass == 0 ? 34 : 20, base = pass == 0 ? 0 : 34;
    for (int q = 0; q <= nq; ++q) {
        double v = q < nq ? loc[q] : cnt;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s[q < nq ? base + q : 54], v);
    }
    __syncthreads();
    if (threadIdx.x < 55) atomicAdd(&acc[threadIdx.x], s[threadIdx.x]);
}

// normalisation constants into the parameter blob (pass 0: xm, xs, ysc;
// pass 1: ym, ys)
__global__ void mlp_norm_kernel(const double* acc, float* w, int pass) {
    const int q = threadIdx.x;
    const double cnt = acc[54] > 0.0 ? acc[54] : 1.0;
    auto dev = [](double sum, double sq, double c) {
        const double mean = sum / c;
        const double var = sq / c - mean * mean;
        return var > 0.0 ? sqrt(var) : 0.0;
    };
    if (pass == 0) {
        if (q < kIn) {
            const double sd = dev(acc[q], acc[kIn + q], cnt);
            w[kOffXm + q] = (float)(acc[q] / cnt);
            w[kOffXs + q] = (float)((sd > 1e-30 && sd < 1e30) ? sd : 1.0);  // a constant input gets a unit scale
        } else if (q < kIn + kOut) {
            // corrections below kMinScale are below the residual the cold
            // start leaves anyway: they map to ~0 and weigh nothing in the loss
            const double g = exp(acc[24 + q - kIn] / cnt);
            w[kOffYsc + q - kIn] = (float)(g > kMinScale ? g : kMinScale);
        }
    } else if (q < kOut) {
        const double sd = dev(acc[34 + q], acc[44 + q], cnt);
        w[kOffYm + q] = (float)(acc[34 + q] / cnt);
        w[kOffYs + q] = (float)(sd > 1.0 && sd < 1e30 ? sd : 1.0);  // at most a unit weight per output
    }
}

// ------------------------------------------------------------------- inference

// One persistent CTA per SM-slot; tiles of 128 fits. Inputs come from the fit
// targets (mode 0: fit 2c uses the moments of f of cell c, fit 2c + 1 the
// fluid moments rescaled by n_V / n_F, as the Newton kernel forms them) or
// from raw inputs (mode 1: x[n][12]). Output: eta* - eta_0 per fit (10
// floats; NaN for fits without usable inputs).
__global__ void __launch_bounds__(kT) mlp_infer_kernel(MlpInferArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sW1 = smem;              // 128 x 16
    unsigned char* sW2 = sW1 + 4096;        // 128 x 128
    unsigned char* sW3 = sW2 + 32768;       // 16 x 128
    unsigned char* sX = sW3 + 4096;         // 128 x 16
    unsigned char* sH = sX + 4096;          // 128 x 128
    __shared__ float sb1[kHid], sb2[kHid], sb3[16], snorm[kNorm];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x;
    const float* w = a.w;
    stage_weights(w, sW1, sW2, sW3, nullptr, nullptr);
    for (int q = t; q < kHid; q += kT) {
        sb1[q] = w[kOffB1 + q];
        sb2[q] = w[kOffB2 + q];
    }
    if (t < 16) sb3[t] = t < kOut ? w[kOffB3 + t] : 0.f;
    if (t < kNorm) snorm[t] = w[t];
    if (t == 0) tc::mbar_init(&bar, 1);
    if (t < 32) tc::tmem_alloc(&tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const int lane0 = 32 * (t >> 5);
    TcState st{&bar, 0u, true};
    for (long long tile = blockIdx.x; tile * kT < a.nfit; tile += gridDim.x) {
        const long long fit = tile * kT + t;
        float x[kIn];
        bool valid = false;
        if (fit < a.nfit) {
            if (a.mode == 1) {
                for (int q = 0; q < kIn; ++q) x[q] = a.x[fit * kIn + q];
                valid = true;
            } else {
                const long long cell = fit >> 1;
                double tg[10];
                const double* vm = a.vmom + cell * a.nmom;
                if ((fit & 1) == 0) {
                    for (int q = 0; q < 10; ++q) tg[q] = vm[q];
                } else {
                    const double nF = a.fluid[cell * 10];
                    const double sc = nF > 0.0 ? vm[0] / nF : 0.0;
                    for (int q = 0; q < 10; ++q) tg[q] = a.fluid[cell * 10 + q] * sc;
                }
                valid = fit_inputs(tg, a.vmin, a.dv, a.vmax, x);
            }
        }
        // a fit whose standardised inputs lie outside the training data
        // (beyond kMaxInputSd standard deviations) gets no warm start
        bool seen = true;
        for (int q = 0; q < 16; ++q) {
            const float v = (valid && q < kIn) ? (x[q] - snorm[kOffXm + q]) / snorm[kOffXs + q] : 0.f;
            seen = seen && fabsf(v) <= kMaxInputSd;
            put_bf16(sX, tc::kmajor_offset(t, q, kT), v);
        }
        if (a.mode == 0) valid = valid && seen;
        // layer 1: Z1 (TMEM columns 0..127)
        st.run([&] { tc::gemm_issue(tmem, sX, sW1, kHid, 16, false); });
        for (int c = 0; c < kHid; c += 16) {
            float v[16];
            tc::tmem_ld16(tc::tmem_at(tmem, lane0, c), v);
            for (int i = 0; i < 16; ++i) put_bf16(sH, tc::kmajor_offset(t, c + i, kT), gelu(v[i] + sb1[c + i]));
        }
        // layer 2: Z2 (columns 128..255)
        st.run([&] { tc::gemm_issue(tmem + 128, sH, sW2, kHid, kHid, false); });
        for (int c = 0; c < kHid; c += 16) {
            float v[16];
            tc::tmem_ld16(tc::tmem_at(tmem, lane0, 128 + c), v);
            for (int i = 0; i < 16; ++i) put_bf16(sH, tc::kmajor_offset(t, c + i, kT), gelu(v[i] + sb2[c + i]));
        }
        // layer 3: Y (columns 0..15)
        st.run([&] { tc::gemm_issue(tmem, sH, sW3, 16, kHid, false); });
        {
            float v[16];
            tc::tmem_ld16(tc::tmem_at(tmem, lane0, 0), v);
            // ... and so does one whose standardised prediction leaves the
            // range of the training targets
            if (a.mode == 0)
                for (int o = 0; o < kOut; ++o) valid = valid && fabsf(v[o] + sb3[o]) <= kMaxOutputSd;
            if (fit < a.nfit)
                for (int o = 0; o < kOut; ++o)
                    a.y[fit * kOut + o] =
                        valid ? snorm[kOffYsc + o] * sinhf((v[o] + sb3[o]) * snorm[kOffYs + o] + snorm[kOffYm + o])
                              : __int_as_float(0x7fc00000);
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    flag_error(a.err, st.ok);
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tmem, 256);
}

// -------------------------------------------------------------------- training

// One training tile: 128 samples (drawn by a counter hash in mode 0, the
// samples row0 + t in mode 1), forward, mean-square loss on the standardised
// transformed outputs, backward; weight and bias gradients are added to a.grad (FP32
// atomics), the loss to a.loss.
__global__ void __launch_bounds__(kT, 1) mlp_train_kernel(MlpTrainArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sW1 = smem;               // 128 x 16
    unsigned char* sW2 = sW1 + 4096;         // 128 x 128
    unsigned char* sW2T = sW2 + 32768;       // 128 x 128
    unsigned char* sW3 = sW2T + 32768;       // 16 x 128
    unsigned char* sW3T = sW3 + 4096;        // 128 x 16
    unsigned char* sX = sW3T + 4096;         // 128 x 16
    unsigned char* sXT = sX + 4096;          // 16 x 128
    unsigned char* bufA = sXT + 4096;        // H1, then H2, then dZ2 (128 x 128)
    unsigned char* bufB = bufA + 32768;      // H1^T
    unsigned char* bufC = bufB + 32768;      // H2^T, then dZ1^T
    unsigned char* bufD = bufC + 32768;      // dZ2^T
    unsigned char* sdY = bufD + 32768;       // 128 x 16
    unsigned char* sdYT = sdY + 4096;        // 16 x 128
    __shared__ float sb1[kHid], sb2[kHid], sb3[16], snorm[kNorm];
    __shared__ float gb1[kHid], gb2[kHid], gb3[16];
    __shared__ double sloss[4];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float* w = a.w;
    stage_weights(w, sW1, sW2, sW3, sW2T, sW3T);
    for (int q = t; q < kHid; q += kT) {
        sb1[q] = w[kOffB1 + q];
        sb2[q] = w[kOffB2 + q];
        gb1[q] = 0.f;
        gb2[q] = 0.f;
    }
    if (t < 16) {
        sb3[t] = t < kOut ? w[kOffB3 + t] : 0.f;
        gb3[t] = 0.f;
    }
    if (t < kNorm) snorm[t] = w[t];
    if (t == 0) tc::mbar_init(&bar, 1);
    if (t < 32) tc::tmem_alloc(&tslot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const int lane0 = 32 * warp;
    TcState st{&bar, 0u, true};

    // ---- the sample of this thread
    const long long row = (long long)blockIdx.x * kT + t;
    long long idx = -1;
    if (a.mode == 0) {
        if (row < a.rows) {
            unsigned long long z = a.seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(row + 1);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            idx = (long long)(z % (unsigned long long)a.n);
        }
    } else {
        const long long r = a.row0 + row;
        if (row < a.rows && r < a.n) idx = r;
    }
    const float* smp = idx >= 0 ? a.samples + idx * kSample : nullptr;
    const bool valid = smp && smp[22] == 1.f;
    for (int q = 0; q < 16; ++q) {
        const float v = (valid && q < kIn) ? (smp[q] - snorm[kOffXm + q]) / snorm[kOffXs + q] : 0.f;
        put_bf16(sX, tc::kmajor_offset(t, q, kT), v);
        put_bf16(sXT, tc::kmajor_offset(q, t, 16), v);
    }
    // ---- forward
    st.run([&] { tc::gemm_issue(tmem, sX, sW1, kHid, 16, false); });  // Z1 -> columns 0..127
    for (int c = 0; c < kHid; c += 16) {
        float v[16];
        tc::tmem_ld16(tc::tmem_at(tmem, lane0, c), v);
        for (int i = 0; i < 16; ++i) {
            const float h = gelu(v[i] + sb1[c + i]);
            put_bf16(bufA, tc::kmajor_offset(t, c + i, kT), h);
            put_bf16(bufB, tc::kmajor_offset(c + i, t, kT), h);
        }
    }
    st.run([&] { tc::gemm_issue(tmem + 128, bufA, sW2, kHid, kHid, false); });  // Z2 -> 128..255
    for (int c = 0; c < kHid; c += 16) {
        float v[16];
        tc::tmem_ld16(tc::tmem_at(tmem, lane0, 128 + c), v);
        for (int i = 0; i < 16; ++i) {
            const float h = gelu(v[i] + sb2[c + i]);
            put_bf16(bufA, tc::kmajor_offset(t, c + i, kT), h);
            put_bf16(bufC, tc::kmajor_offset(c + i, t, kT), h);
        }
    }
    st.run([&] { tc::gemm_issue(tmem + 256, bufA, sW3, 16, kHid, false); });  // Y -> 256..271
    double lsum = 0.0;
    {
        float v[16];
        tc::tmem_ld16(tc::tmem_at(tmem, lane0, 256), v);
        for (int o = 0; o < 16; ++o) {
            float d = 0.f;
            if (valid && o < kOut) {
                const float ts = (asinhf(smp[kIn + o] / snorm[kOffYsc + o]) - snorm[kOffYm + o]) / snorm[kOffYs + o];
                const float diff = v[o] + sb3[o] - ts;
                lsum += (double)diff * diff;
                d = 2.f * diff * a.inv_count;
            }
            put_bf16(sdY, tc::kmajor_offset(t, o, kT), d);
            put_bf16(sdYT, tc::kmajor_offset(o, t, 16), d);
            float r = d;
            for (int s = 16; s > 0; s >>= 1) r += __shfl_xor_sync(kAll, r, s);
            if (lane == 0 && o < kOut) atomicAdd_block(&gb3[o], r);
        }
    }
    // ---- backward: dH2 = dY W3 (columns 256..383), dZ2 = dH2 * gelu'(Z2)
    st.run([&] { tc::gemm_issue(tmem + 256, sdY, sW3T, kHid, 16, false); });
    for (int c = 0; c < kHid; c += 16) {
        float g[16], z[16];
        tc::tmem_ld16(tc::tmem_at(tmem, lane0, 256 + c), g);
        tc::tmem_ld16(tc::tmem_at(tmem, lane0, 128 + c), z);
        for (int i = 0; i < 16; ++i) {
            const float d = g[i] * gelu_grad(z[i] + sb2[c + i]);
            put_bf16(bufA, tc::kmajor_offset(t, c + i, kT), d);
            put_bf16(bufD, tc::kmajor_offset(c + i, t, kT), d);
            float r = d;
            for (int s = 16; s > 0; s >>= 1) r += __shfl_xor_sync(kAll, r, s);
            if (lane == 0) atomicAdd_block(&gb2[c + i], r);
        }
    }
    // dW3^T = H2^T dY (columns 384..399) and dW2 = dZ2^T H1 (columns 256..383)
    st.run([&] {
        tc::gemm_issue(tmem + 384, bufC, sdYT, 16, kT, false);
        tc::gemm_issue(tmem + 256, bufD, bufB, kHid, kT, false);
    });
    {
        float v[16];
        tc::tmem_ld16(tc::tmem_at(tmem, lane0, 384), v);  // row t = hidden unit t of layer 2's output
        for (int o = 0; o < kOut; ++o) atomicAdd(&a.grad[kOffW3 + o * kHid + t], v[o]);
        for (int c = 0; c < kHid; c += 16) {
            tc::tmem_ld16(tc::tmem_at(tmem, lane0, 256 + c), v);  // row t = output unit t of layer 2
            for (int i = 0; i < 16; ++i) atomicAdd(&a.grad[kOffW2 + t * kHid + c + i], v[i]);
        }
    }
    // dH1 = dZ2 W2 (columns 256..383), dZ1 = dH1 * gelu'(Z1) -> bufC (transposed)
    st.run([&] { tc::gemm_issue(tmem + 256, bufA, sW2T, kHid, kHid, false); });
    for (int c = 0; c < kHid; c += 16) {
        float g[16], z[16];
        tc::tmem_ld16(tc::tmem_at(tmem, lane0, 256 + c), g);
        tc::tmem_ld16(tc::tmem_at(tmem, lane0, c), z);
        for (int i = 0; i < 16; ++i) {
            const float d = g[i] * gelu_grad(z[i] + sb1[c + i]);
            put_bf16(bufC, tc::kmajor_offset(c + i, t, kT), d);
            float r = d;
            for (int s = 16; s > 0; s >>= 1) r += __shfl_xor_sync(kAll, r, s);
            if (lane == 0) atomicAdd_block(&gb1[c + i], r);
        }
    }
    // dW1 = dZ1^T X (columns 384..399)
    st.run([&] { tc::gemm_issue(tmem + 384, bufC, sXT, 16, kT, false); });
    {
        float v[16];
        tc::tmem_ld16(tc::tmem_at(tmem, lane0, 384), v);  // row t = hidden unit t of layer 1
        for (int i = 0; i < kIn; ++i) atomicAdd(&a.grad[kOffW1 + t * kIn + i], v[i]);
    }
    // biases and loss
    for (int s = 16; s > 0; s >>= 1) lsum += __shfl_xor_sync(kAll, lsum, s);
    if (lane == 0) sloss[warp] = lsum;
    tc::fence_before_sync();
    __syncthreads();
    atomicAdd(&a.grad[kOffB1 + t], gb1[t]);
    atomicAdd(&a.grad[kOffB2 + t], gb2[t]);
    if (t < kOut) atomicAdd(&a.grad[kOffB3 + t], gb3[t]);
    if (t == 0) atomicAdd(a.loss, sloss[0] + sloss[1] + sloss[2] + sloss[3]);
    flag_error(a.err, st.ok);
    if (t < 32) tc::tmem_dealloc(tmem, 512);
}

// Adam on the trained parameters (FP32 master weights)
__global__ void mlp_adam_kernel(float* w, float* m, float* v, const float* g, float lr, float b1, float b2,
                                float c1, float c2) {
    const int i = kFirstTrained + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParam) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// ------------------------------------------------------------------- launchers

static constexpr size_t kInferSmem = 4096 + 32768 + 4096 + 4096 + 32768;
static constexpr size_t kTrainSmem = 4096 + 32768 * 2 + 4096 * 4 + 32768 * 4 + 4096 * 2;

static int mlp_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

cudaError_t launch_mlp_stats(const float* samples, long long n, double* acc, float* w, cudaStream_t st) {
    long long blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    for (int pass = 0; pass < 2; ++pass) {
        cudaError_t e = cudaMemsetAsync(acc, 0, 55 * sizeof(double), st);
        if (e != cudaSuccess) return e;
        mlp_stats_kernel<<<(unsigned)blocks, 256, 0, st>>>(samples, n, w, pass, acc);
        mlp_norm_kernel<<<1, 32, 0, st>>>(acc, w, pass);
        count_launch(2);
    }
    return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const MlpInferArgs& a, cudaStream_t st) {
    if (a.nfit <= 0) return cudaSuccess;
    cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInferSmem);
    long long tiles = (a.nfit + kT - 1) / kT;
    long long grid = (long long)mlp_sms() * 2;  // two CTAs (2 x 256 TMEM columns) per SM
    if (grid > tiles) grid = tiles;
    mlp_infer_kernel<<<(unsigned)grid, kT, kInferSmem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_train_step(const MlpTrainArgs& a, cudaStream_t st) {
    cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
    const long long grid = (a.rows + kT - 1) / kT;
    if (grid <= 0) return cudaSuccess;
    mlp_train_kernel<<<(unsigned)grid, kT, kTrainSmem, st>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* w, float* m, float* v, const float* g, float lr, int step, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    const int n = kNParam - kFirstTrained;
    mlp_adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(w, m, v, g, lr, b1, b2, c1, c2);
    count_launch();
    return cudaGetLastError();
}

}  // namespace vl
