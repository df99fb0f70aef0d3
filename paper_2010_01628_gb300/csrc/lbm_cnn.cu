// lbm_cnn.cu -- learned warm start: a small 3D convolutional network that maps
// (Reynolds number, node coordinates, lid mask) to the steady (rho, u) of the
// lid-driven cavity, trained on steady states produced by the solver; its
// prediction initialises the populations (f = f_eq of the predicted fields).
//
// Architecture (fixed): 4 layers of 3x3x3 convolutions with zero padding,
// 5 -> 32 -> 32 -> 32 -> 4 channels, ReLU after the first three.  Activations
// and the weights used by the kernels are BF16 (channel-last, channels padded
// to multiples of 16); master weights, gradients and Adam moments are FP32.
//
// Kernels:
//  - conv_mma: implicit GEMM on the tensor cores (mma.sync m16n8k16 BF16 with
//    FP32 accumulation).  A warp computes 64 voxels x all output channels;
//    the 27 taps x input channels form the reduction.  The same kernel runs the
//    backward data pass with the flipped, transposed weights.
//  - conv_wgrad: weight and bias gradients, FP32 reductions over voxel chunks
//    (one partial per CTA, summed in a fixed order).
//  - adam: the optimiser step on the FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_internal.h"

namespace cnn {

constexpr int NL = 4;
constexpr int C_IN_REAL = 5, C_OUT_REAL = 4;
// padded channel counts per layer boundary: input 16, hidden 32, output 16
constexpr int CH[NL + 1] = {16, 32, 32, 32, 16};
constexpr int CH_REAL[NL + 1] = {5, 32, 32, 32, 4};
constexpr float RHO_SCALE = 30.f;  // network output 0 = (rho - 1) * RHO_SCALE
constexpr float U_SCALE = 10.f;    // outputs 1..3 = u * U_SCALE (lid speed 0.1 -> 1)
constexpr int WG_BLOCKS = 304;     // CTAs of the weight-gradient reduction

constexpr int layer_params(int l) { return 27 * CH_REAL[l + 1] * CH_REAL[l] + CH_REAL[l + 1]; }
constexpr int total_params() { return layer_params(0) + layer_params(1) + layer_params(2) + layer_params(3); }

struct Shape {
    int nx, ny, nz;
    long P;
};

__device__ __forceinline__ void tap_offset(int tap, int& dx, int& dy, int& dz) {
    dx = tap % 3 - 1;
    dy = (tap / 3) % 3 - 1;
    dz = tap / 9 - 1;
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t bf_pack(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// EPI: 0 = +bias, ReLU, BF16 out; 1 = +bias, FP32 out; 2 = ReLU mask from
// `gate` (the forward activation of this layer's output), BF16 out, no bias.
template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(128) conv_mma(const __nv_bfloat16* __restrict__ X,
                                                const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ bias,
                                                void* __restrict__ Y, const __nv_bfloat16* __restrict__ gate,
                                                Shape s) {
    extern __shared__ __align__(16) uint32_t wsm[];  // [27][CO][CI/2] packed bf16 pairs
    constexpr int NT = CO / 8, KS = CI / 16;
    for (int i = threadIdx.x; i < 27 * CO * CI / 2; i += blockDim.x) wsm[i] = reinterpret_cast<const uint32_t*>(Wt)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long base = ((long)blockIdx.x * 4 + warp) * 64;
    const int r = lane >> 2, q = lane & 3;
    const uint32_t* X32 = reinterpret_cast<const uint32_t*>(X);
    // the 8 voxels this thread loads A rows for: rows r and r+8 of 4 m-tiles
    int vx[8], vy[8], vz[8];
    bool vin[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const long p = base + (j >> 1) * 16 + r + (j & 1) * 8;
        vin[j] = p < s.P;
        const long pp = vin[j] ? p : 0;
        vx[j] = (int)(pp % s.nx);
        vy[j] = (int)((pp / s.nx) % s.ny);
        vz[j] = (int)(pp / ((long)s.nx * s.ny));
    }
    float acc[4][NT][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[m][n][k] = 0.f;
    for (int tap = 0; tap < 27; ++tap) {
        int dx, dy, dz;
        tap_offset(tap, dx, dy, dz);
        long src[8];
        bool ok[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int x = vx[j] + dx, y = vy[j] + dy, z = vz[j] + dz;
            ok[j] = vin[j] && x >= 0 && x < s.nx && y >= 0 && y < s.ny && z >= 0 && z < s.nz;
            src[j] = ok[j] ? (((long)z * s.ny + y) * s.nx + x) * (CI / 2) : 0;
        }
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const int k0 = ks * 8 + q;  // packed-pair index of channels 2q, 2q+1 within this k-step
            uint32_t a[4][4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                a[m][0] = ok[2 * m] ? __ldg(X32 + src[2 * m] + k0) : 0u;
                a[m][1] = ok[2 * m + 1] ? __ldg(X32 + src[2 * m + 1] + k0) : 0u;
                a[m][2] = ok[2 * m] ? __ldg(X32 + src[2 * m] + k0 + 4) : 0u;
                a[m][3] = ok[2 * m + 1] ? __ldg(X32 + src[2 * m + 1] + k0 + 4) : 0u;
            }
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const uint32_t* wrow = wsm + ((size_t)tap * CO + n * 8 + r) * (CI / 2) + k0;
                const uint32_t b0 = wrow[0], b1 = wrow[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) mma_bf16(acc[m][n], a[m], b0, b1);
            }
        }
    }
    // epilogue: D rows r (c0, c1) and r + 8 (c2, c3), columns n*8 + 2q, +1
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long p = base + m * 16 + r + h * 8;
            if (p >= s.P) continue;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int co = n * 8 + 2 * q;
                float v0 = acc[m][n][2 * h], v1 = acc[m][n][2 * h + 1];
                if (EPI == 0 || EPI == 1) {
                    v0 += bias[co];
                    v1 += bias[co + 1];
                }
                if (EPI == 0) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (EPI == 2) {
                    const uint32_t g = reinterpret_cast<const uint32_t*>(gate)[p * (CO / 2) + co / 2];
                    if (!(bf_lo(g) > 0.f)) v0 = 0.f;
                    if (!(bf_hi(g) > 0.f)) v1 = 0.f;
                }
                if (EPI == 1) {
                    float* Yf = reinterpret_cast<float*>(Y);
                    Yf[p * CO + co] = v0;
                    Yf[p * CO + co + 1] = v1;
                } else {
                    reinterpret_cast<uint32_t*>(Y)[p * (CO / 2) + co / 2] = bf_pack(v0, v1);
                }
            }
        }
}

// Weight/bias gradients: dW[tap][co][ci] = sum_p dY[p][co] X[p + off(tap)][ci],
// db[co] = sum_p dY[p][co].  256 threads: thread (co = t % 32, group g = t / 32)
// accumulates taps g, g+8, g+16, g+24 for all CI; one partial per CTA.
template <int CI, int CO>
__global__ void __launch_bounds__(256) conv_wgrad(const __nv_bfloat16* __restrict__ X,
                                                  const __nv_bfloat16* __restrict__ dY, float* __restrict__ partial,
                                                  Shape s) {
    const int co = threadIdx.x & 31, g = threadIdx.x >> 5;
    const bool co_ok = co < CO;
    float acc[4][CI];
    float db = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int c = 0; c < CI; ++c) acc[t][c] = 0.f;
    const long chunk = (s.P + gridDim.x - 1) / gridDim.x;
    const long p0 = blockIdx.x * chunk, p1 = min(s.P, p0 + chunk);
    const unsigned short* dYs = reinterpret_cast<const unsigned short*>(dY);
    const uint4* X4 = reinterpret_cast<const uint4*>(X);
    for (long p = p0; p < p1; ++p) {
        const float gy = co_ok ? __uint_as_float((uint32_t)__ldg(dYs + p * CO + co) << 16) : 0.f;
        db += gy;
        const int x = (int)(p % s.nx), y = (int)((p / s.nx) % s.ny), z = (int)(p / ((long)s.nx * s.ny));
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int tap = g + 8 * t;
            if (tap >= 27) continue;
            int dx, dy, dz;
            tap_offset(tap, dx, dy, dz);
            const int xs = x + dx, ys = y + dy, zs = z + dz;
            if (xs < 0 || xs >= s.nx || ys < 0 || ys >= s.ny || zs < 0 || zs >= s.nz) continue;
            const long q = ((long)zs * s.ny + ys) * s.nx + xs;
#pragma unroll
            for (int v = 0; v < CI / 8; ++v) {
                const uint4 w = __ldg(X4 + q * (CI / 8) + v);
                acc[t][8 * v + 0] += gy * bf_lo(w.x);
                acc[t][8 * v + 1] += gy * bf_hi(w.x);
                acc[t][8 * v + 2] += gy * bf_lo(w.y);
                acc[t][8 * v + 3] += gy * bf_hi(w.y);
                acc[t][8 * v + 4] += gy * bf_lo(w.z);
                acc[t][8 * v + 5] += gy * bf_hi(w.z);
                acc[t][8 * v + 6] += gy * bf_lo(w.w);
                acc[t][8 * v + 7] += gy * bf_hi(w.w);
            }
        }
    }
    // partial layout per CTA: [27][CO][CI] then [CO] biases
    float* out = partial + (size_t)blockIdx.x * (27 * CO * CI + CO);
    if (co_ok) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int tap = g + 8 * t;
            if (tap >= 27) continue;
#pragma unroll
            for (int c = 0; c < CI; ++c) out[((size_t)tap * CO + co) * CI + c] = acc[t][c];
        }
        if (g == 0) out[27 * CO * CI + co] = db;
    }
}

__global__ void sum_partials(const float* __restrict__ partial, int nblocks, int width, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= width) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * width + i];
    out[i] = s;
}

// Master weights of layer l: [CO_real][CI_real][27] then bias [CO_real].
// Pack to the kernel layouts: fwd [27][CO][CI] and bwd-data [27][CI][CO]
// with the tap flipped (26 - tap); padding channels are zero.
__global__ void pack_weights(const float* __restrict__ master, __nv_bfloat16* __restrict__ wf,
                             __nv_bfloat16* __restrict__ wb, float* __restrict__ bias, int ci_r, int co_r, int ci_p,
                             int co_p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = 27 * co_p * ci_p;
    if (i < n) {
        const int tap = i / (co_p * ci_p), co = (i / ci_p) % co_p, ci = i % ci_p;
        const float v = (co < co_r && ci < ci_r) ? master[((size_t)co * ci_r + ci) * 27 + tap] : 0.f;
        wf[i] = __float2bfloat16_rn(v);
        wb[((size_t)(26 - tap) * ci_p + ci) * co_p + co] = __float2bfloat16_rn(v);
    }
    if (i < co_p) bias[i] = i < co_r ? master[(size_t)27 * co_r * ci_r + i] : 0.f;
}

// Gather the padded per-layer gradient into the master layout.
__global__ void unpack_grad(const float* __restrict__ g, float* __restrict__ master_grad, int ci_r, int co_r, int ci_p,
                            int co_p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = co_r * ci_r * 27;
    if (i < n) {
        const int co = i / (ci_r * 27), ci = (i / 27) % ci_r, tap = i % 27;
        master_grad[i] = g[((size_t)tap * co_p + co) * ci_p + ci];
    }
    if (i < co_r) master_grad[n + i] = g[(size_t)27 * co_p * ci_p + i];
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Input channels: [Re_n, x_n, y_n, z_n, lid] (+ zero padding to 16);
// Re_n = (Re - 550)/450, coordinates of node centres scaled to [-1, 1], lid = 1
// on the top (+y) layer of nodes.
__global__ void features(__nv_bfloat16* __restrict__ X0, Shape s, float re_n) {
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.P) return;
    const int x = (int)(p % s.nx), y = (int)((p / s.nx) % s.ny), z = (int)(p / ((long)s.nx * s.ny));
    float f[16] = {0};
    f[0] = re_n;
    f[1] = 2.f * (x + 0.5f) / s.nx - 1.f;
    f[2] = 2.f * (y + 0.5f) / s.ny - 1.f;
    f[3] = 2.f * (z + 0.5f) / s.nz - 1.f;
    f[4] = y == s.ny - 1 ? 1.f : 0.f;
    uint32_t* o = reinterpret_cast<uint32_t*>(X0) + p * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = bf_pack(f[2 * k], f[2 * k + 1]);
}

// Loss and its gradient: L = mean over voxels and the 4 real channels of
// (Y - T)^2 with T = [(rho - 1) RHO_SCALE, u U_SCALE] from FP64 fields.
__global__ void loss_grad(const float* __restrict__ Y, const double* __restrict__ rho, const double* __restrict__ u,
                          __nv_bfloat16* __restrict__ dY, double* __restrict__ partial, Shape s) {
    __shared__ double sh[256];
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (p < s.P) {
        const float t[4] = {(float)((rho[p] - 1.0) * RHO_SCALE), (float)(u[p] * U_SCALE), (float)(u[s.P + p] * U_SCALE),
                            (float)(u[2 * s.P + p] * U_SCALE)};
        const float scale = 2.f / (4.f * (float)s.P);
        float d[16] = {0};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float e = Y[p * 16 + c] - t[c];
            l += (double)e * e;
            d[c] = scale * e;
        }
        uint32_t* o = reinterpret_cast<uint32_t*>(dY) + p * 8;
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = bf_pack(d[2 * k], d[2 * k + 1]);
    }
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void sum_double(const double* __restrict__ partial, long n, double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// Prediction -> FP64 fields rho = 1 + y0/RHO_SCALE, u = y1..3/U_SCALE (planar).
__global__ void to_fields(const float* __restrict__ Y, double* __restrict__ rho, double* __restrict__ u, Shape s) {
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.P) return;
    rho[p] = 1.0 + (double)Y[p * 16 + 0] / RHO_SCALE;
    u[p] = (double)Y[p * 16 + 1] / U_SCALE;
    u[s.P + p] = (double)Y[p * 16 + 2] / U_SCALE;
    u[2 * s.P + p] = (double)Y[p * 16 + 3] / U_SCALE;
}

}  // namespace cnn

struct lbm_cnn {
    cnn::Shape s;
    cudaStream_t stream;
    lbm_alloc_fn alloc;
    lbm_free_fn release;
    void* user;
    float* master;    // FP32 master weights, all layers back to back
    float* grad;      // FP32 gradient, same layout
    float* adam_m;
    float* adam_v;
    long adam_t = 0;
    __nv_bfloat16* wf[cnn::NL];  // packed BF16 forward weights
    __nv_bfloat16* wb[cnn::NL];  // packed BF16 backward-data weights
    float* bias[cnn::NL];
    float* gpad[cnn::NL];        // padded per-layer gradient (summed partials)
    float* partial;              // weight-gradient partials
    __nv_bfloat16* act[cnn::NL]; // act[0] = input features, act[1..3] hidden activations
    float* out;                  // [P][16] FP32 prediction
    __nv_bfloat16* dA[2];        // backward activations (ping-pong)
    double* rho_d;               // FP64 fields (prediction or target staging)
    double* u_d;
    double* lpart;               // loss partials
    double* lsum;
    std::string err;
};

namespace {

void* cnn_alloc(lbm_cnn* c, size_t bytes) {
    if (c->alloc) return c->alloc(bytes, (void*)c->stream, c->user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void cnn_free(lbm_cnn* c, void* p) {
    if (!p) return;
    if (c->release)
        c->release(p, (void*)c->stream, c->user);
    else
        cudaFree(p);
}

size_t layer_offset(int l) {
    size_t o = 0;
    for (int k = 0; k < l; ++k) o += (size_t)cnn::layer_params(k);
    return o;
}

template <int CI, int CO, int EPI>
cudaError_t conv(lbm_cnn* c, const __nv_bfloat16* X, const __nv_bfloat16* W, const float* bias, void* Y,
                 const __nv_bfloat16* gate) {
    const size_t smem = (size_t)27 * CO * CI * 2;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(cnn::conv_mma<CI, CO, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const long blocks = (c->s.P + 255) / 256;
    cnn::conv_mma<CI, CO, EPI><<<(unsigned)blocks, 128, smem, c->stream>>>(X, W, bias, Y, gate, c->s);
    return cudaGetLastError();
}

template <int CI, int CO>
cudaError_t wgrad(lbm_cnn* c, const __nv_bfloat16* X, const __nv_bfloat16* dY, float* gpad) {
    cnn::conv_wgrad<CI, CO><<<cnn::WG_BLOCKS, 256, 0, c->stream>>>(X, dY, c->partial, c->s);
    const int width = 27 * CO * CI + CO;
    cnn::sum_partials<<<(width + 255) / 256, 256, 0, c->stream>>>(c->partial, cnn::WG_BLOCKS, width, gpad);
    return cudaGetLastError();
}

cudaError_t pack_all(lbm_cnn* c) {
    for (int l = 0; l < cnn::NL; ++l) {
        const int ci_p = cnn::CH[l], co_p = cnn::CH[l + 1];
        const int n = 27 * ci_p * co_p;
        cnn::pack_weights<<<(n + 255) / 256, 256, 0, c->stream>>>(c->master + layer_offset(l), c->wf[l], c->wb[l],
                                                                   c->bias[l], cnn::CH_REAL[l], cnn::CH_REAL[l + 1],
                                                                   ci_p, co_p);
    }
    return cudaGetLastError();
}

cudaError_t forward(lbm_cnn* c) {
    cudaError_t e = conv<16, 32, 0>(c, c->act[0], c->wf[0], c->bias[0], c->act[1], nullptr);
    if (e == cudaSuccess) e = conv<32, 32, 0>(c, c->act[1], c->wf[1], c->bias[1], c->act[2], nullptr);
    if (e == cudaSuccess) e = conv<32, 32, 0>(c, c->act[2], c->wf[2], c->bias[2], c->act[3], nullptr);
    if (e == cudaSuccess) e = conv<32, 16, 1>(c, c->act[3], c->wf[3], c->bias[3], c->out, nullptr);
    return e;
}

// Backward from dY4 (held in dA[1] reinterpreted as [P][16]); fills c->grad.
cudaError_t backward(lbm_cnn* c, const __nv_bfloat16* dY4) {
    cudaError_t e = wgrad<32, 16>(c, c->act[3], dY4, c->gpad[3]);
    // dA3 = conv^T(dY4, W4) masked by act3 > 0
    if (e == cudaSuccess) e = conv<16, 32, 2>(c, dY4, c->wb[3], nullptr, c->dA[0], c->act[3]);
    if (e == cudaSuccess) e = wgrad<32, 32>(c, c->act[2], c->dA[0], c->gpad[2]);
    if (e == cudaSuccess) e = conv<32, 32, 2>(c, c->dA[0], c->wb[2], nullptr, c->dA[1], c->act[2]);
    if (e == cudaSuccess) e = wgrad<32, 32>(c, c->act[1], c->dA[1], c->gpad[1]);
    if (e == cudaSuccess) e = conv<32, 32, 2>(c, c->dA[1], c->wb[1], nullptr, c->dA[0], c->act[1]);
    if (e == cudaSuccess) e = wgrad<16, 32>(c, c->act[0], c->dA[0], c->gpad[0]);
    for (int l = 0; l < cnn::NL && e == cudaSuccess; ++l) {
        const int n = 27 * cnn::CH_REAL[l] * cnn::CH_REAL[l + 1];
        cnn::unpack_grad<<<(n + 255) / 256, 256, 0, c->stream>>>(c->gpad[l], c->grad + layer_offset(l),
                                                                  cnn::CH_REAL[l], cnn::CH_REAL[l + 1], cnn::CH[l],
                                                                  cnn::CH[l + 1]);
        e = cudaGetLastError();
    }
    return e;
}

// Loss against FP64 target fields (device, planar rho [P], u [3P]); writes
// dY4 into its buffer and the loss sum into c->lsum.
cudaError_t loss(lbm_cnn* c, const double* rho, const double* u, __nv_bfloat16* dY4) {
    const long blocks = (c->s.P + 255) / 256;
    cnn::loss_grad<<<(unsigned)blocks, 256, 0, c->stream>>>(c->out, rho, u, dY4, c->lpart, c->s);
    cnn::sum_double<<<1, 256, 0, c->stream>>>(c->lpart, blocks, c->lsum);
    return cudaGetLastError();
}

lbm_status cnn_cuda_fail(lbm_cnn* c, cudaError_t e, const char* where) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    c->err = buf;
    return LBM_ERR_CUDA;
}

// Stage FP64 target fields (host or device pointers) into the CNN's buffers.
cudaError_t stage_fields(lbm_cnn* c, const double* rho, const double* u) {
    const size_t P = (size_t)c->s.P;
    cudaError_t e = cudaMemcpyAsync(c->rho_d, rho, P * 8, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->u_d, u, 3 * P * 8, cudaMemcpyDefault, c->stream);
    return e;
}

}  // namespace

extern "C" {

size_t lbm_cnn_param_count(void) { return (size_t)cnn::total_params(); }

lbm_status lbm_cnn_create(lbm_cnn** out, int nx, int ny, int nz, const float* init_weights, void* cuda_stream) {
    if (!out || nx < 1 || ny < 1 || nz < 1) return LBM_ERR_ARG;
    *out = nullptr;
    const double P = (double)nx * ny * nz;
    if (P > 268435456.0) return LBM_ERR_ARG;  // 2^28 voxels
    lbm_cnn* c = new (std::nothrow) lbm_cnn();
    if (!c) return LBM_ERR_OOM;
    lbm_alloc_fn a;
    lbm_free_fn r;
    void* u;
    lbm_internal_get_allocator(&a, &r, &u);
    c->alloc = a;
    c->release = r;
    c->user = u;
    c->s.nx = nx;
    c->s.ny = ny;
    c->s.nz = nz;
    c->s.P = (long)nx * ny * nz;
    c->stream = (cudaStream_t)cuda_stream;
    const size_t NP = lbm_cnn_param_count();
    const size_t Pn = (size_t)c->s.P;
    bool ok = true;
    auto A = [&](size_t bytes) {
        void* p = cnn_alloc(c, bytes);
        ok = ok && p;
        return p;
    };
    c->master = (float*)A(NP * 4);
    c->grad = (float*)A(NP * 4);
    c->adam_m = (float*)A(NP * 4);
    c->adam_v = (float*)A(NP * 4);
    size_t maxw = 0;
    for (int l = 0; l < cnn::NL; ++l) {
        const size_t w = (size_t)27 * cnn::CH[l] * cnn::CH[l + 1];
        c->wf[l] = (__nv_bfloat16*)A(w * 2);
        c->wb[l] = (__nv_bfloat16*)A(w * 2);
        c->bias[l] = (float*)A((size_t)cnn::CH[l + 1] * 4);
        c->gpad[l] = (float*)A((w + cnn::CH[l + 1]) * 4);
        maxw = std::max(maxw, w + (size_t)cnn::CH[l + 1]);
        c->act[l] = (__nv_bfloat16*)A(Pn * cnn::CH[l] * 2);
    }
    c->partial = (float*)A((size_t)cnn::WG_BLOCKS * maxw * 4);
    c->out = (float*)A(Pn * 16 * 4);
    c->dA[0] = (__nv_bfloat16*)A(Pn * 32 * 2);
    c->dA[1] = (__nv_bfloat16*)A(Pn * 32 * 2);
    c->rho_d = (double*)A(Pn * 8);
    c->u_d = (double*)A(3 * Pn * 8);
    c->lpart = (double*)A(((Pn + 255) / 256) * 8);
    c->lsum = (double*)A(8);
    if (!ok) {
        lbm_cnn_destroy(c);
        return LBM_ERR_OOM;
    }
    cudaError_t e = cudaSuccess;
    if (init_weights) {
        e = cudaMemcpyAsync(c->master, init_weights, NP * 4, cudaMemcpyDefault, c->stream);
    } else {
        // He-uniform initialisation from a fixed LCG (deterministic)
        std::vector<float> w(NP);
        unsigned long long st = 0x9E3779B97F4A7C15ull;
        size_t o = 0;
        for (int l = 0; l < cnn::NL; ++l) {
            const int fan_in = 27 * cnn::CH_REAL[l];
            const float lim = std::sqrt(6.0f / fan_in);
            const int nw = 27 * cnn::CH_REAL[l] * cnn::CH_REAL[l + 1];
            for (int i = 0; i < nw; ++i) {
                st = st * 6364136223846793005ull + 1442695040888963407ull;
                const float r01 = (float)((st >> 40) & 0xFFFFFF) / 16777216.0f;
                w[o + i] = (2.f * r01 - 1.f) * lim;
            }
            for (int i = 0; i < cnn::CH_REAL[l + 1]; ++i) w[o + nw + i] = 0.f;
            o += (size_t)cnn::layer_params(l);
        }
        e = cudaMemcpyAsync(c->master, w.data(), NP * 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->adam_m, 0, NP * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->adam_v, 0, NP * 4, c->stream);
    for (int l = 0; l < cnn::NL && e == cudaSuccess; ++l)
        e = cudaMemsetAsync(c->act[l], 0, Pn * cnn::CH[l] * 2, c->stream);
    if (e == cudaSuccess) e = pack_all(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        lbm_cnn_destroy(c);
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    *out = c;
    return LBM_OK;
}

void lbm_cnn_destroy(lbm_cnn* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    void* ptrs[] = {c->master, c->grad,  c->adam_m, c->adam_v, c->partial, c->out, c->dA[0],
                    c->dA[1],  c->rho_d, c->u_d,    c->lpart,  c->lsum};
    for (void* p : ptrs) cnn_free(c, p);
    for (int l = 0; l < cnn::NL; ++l) {
        cnn_free(c, c->wf[l]);
        cnn_free(c, c->wb[l]);
        cnn_free(c, c->bias[l]);
        cnn_free(c, c->gpad[l]);
        cnn_free(c, c->act[l]);
    }
    delete c;
}

const char* lbm_cnn_last_error(const lbm_cnn* c) { return c ? c->err.c_str() : "null network"; }

lbm_status lbm_cnn_set_weights(lbm_cnn* c, const float* w, size_t count) {
    if (!c || !w || count != lbm_cnn_param_count()) return LBM_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(c->master, w, count * 4, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = pack_all(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_set_weights");
}

lbm_status lbm_cnn_get_weights(lbm_cnn* c, float* w, size_t count) {
    if (!c || !w || count != lbm_cnn_param_count()) return LBM_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(w, c->master, count * 4, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_get_weights");
}

lbm_status lbm_cnn_set_input(lbm_cnn* c, double reynolds) {
    if (!c) return LBM_ERR_ARG;
    const long blocks = (c->s.P + 255) / 256;
    cnn::features<<<(unsigned)blocks, 256, 0, c->stream>>>(c->act[0], c->s, (float)((reynolds - 550.0) / 450.0));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_set_input");
}

lbm_status lbm_cnn_set_input_raw(lbm_cnn* c, const float* x, size_t count) {
    // x: [P][5] FP32 input channels (host or device); padded to BF16 [P][16]
    if (!c || !x || count != (size_t)c->s.P * cnn::C_IN_REAL) return LBM_ERR_ARG;
    std::vector<float> h((size_t)c->s.P * 16, 0.f);
    std::vector<float> in(count);
    cudaError_t e = cudaMemcpy(in.data(), x, count * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return cnn_cuda_fail(c, e, "lbm_cnn_set_input_raw");
    std::vector<__nv_bfloat16> hb((size_t)c->s.P * 16);
    for (long p = 0; p < c->s.P; ++p)
        for (int k = 0; k < 16; ++k) hb[p * 16 + k] = __float2bfloat16_rn(k < 5 ? in[p * 5 + k] : 0.f);
    e = cudaMemcpyAsync(c->act[0], hb.data(), hb.size() * 2, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_set_input_raw");
}

lbm_status lbm_cnn_forward(lbm_cnn* c, float* out, size_t count) {
    // out (optional): [P][4] FP32 prediction (host or device)
    if (!c) return LBM_ERR_ARG;
    if (out && count != (size_t)c->s.P * cnn::C_OUT_REAL) return LBM_ERR_ARG;
    cudaError_t e = forward(c);
    if (e == cudaSuccess && out)
        e = cudaMemcpy2DAsync(out, 4 * sizeof(float), c->out, 16 * sizeof(float), 4 * sizeof(float), (size_t)c->s.P,
                              cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_forward");
}

lbm_status lbm_cnn_gradient(lbm_cnn* c, const double* rho, const double* u, double* loss_out, float* grad_out,
                            size_t count) {
    if (!c || !rho || !u) return LBM_ERR_ARG;
    if (grad_out && count != lbm_cnn_param_count()) return LBM_ERR_ARG;
    cudaError_t e = stage_fields(c, rho, u);
    if (e == cudaSuccess) e = forward(c);
    __nv_bfloat16* dY4 = c->dA[1];
    if (e == cudaSuccess) e = loss(c, c->rho_d, c->u_d, dY4);
    if (e == cudaSuccess) e = backward(c, dY4);
    double l = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, c->lsum, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, c->grad, count * 4, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cnn_cuda_fail(c, e, "lbm_cnn_gradient");
    if (loss_out) *loss_out = l / (4.0 * (double)c->s.P);
    return LBM_OK;
}

lbm_status lbm_cnn_train_step(lbm_cnn* c, const double* rho, const double* u, float lr, double* loss_out) {
    lbm_status st = lbm_cnn_gradient(c, rho, u, loss_out, nullptr, 0);
    if (st != LBM_OK) return st;
    const int n = (int)lbm_cnn_param_count();
    c->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)c->adam_t)), c2 = 1.f / (1.f - std::pow(b2, (float)c->adam_t));
    cnn::adam_kernel<<<(n + 255) / 256, 256, 0, c->stream>>>(c->master, c->adam_m, c->adam_v, c->grad, n, lr, b1, b2,
                                                              1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = pack_all(c);
    return e == cudaSuccess ? LBM_OK : cnn_cuda_fail(c, e, "lbm_cnn_train_step");
}

lbm_status lbm_cnn_warm_start(lbm_cnn* c, lbm_ctx* ctx, double reynolds) {
    if (!c || !ctx) return LBM_ERR_ARG;
    lbm_status st = lbm_cnn_set_input(c, reynolds);
    if (st != LBM_OK) return st;
    cudaError_t e = forward(c);
    const long blocks = (c->s.P + 255) / 256;
    if (e == cudaSuccess) {
        cnn::to_fields<<<(unsigned)blocks, 256, 0, c->stream>>>(c->out, c->rho_d, c->u_d, c->s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cnn_cuda_fail(c, e, "lbm_cnn_warm_start");
    return lbm_init_fields(ctx, c->rho_d, c->u_d, nullptr, nullptr);
}

}  // extern "C"
