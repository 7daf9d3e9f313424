// unet_kernels.cu -- kernels of the learned warm start: a U-Net that maps a
// porous mask (plus tau and an x ramp) to the normalised steady fields
// (rho - rho_out)/drho and u nu (N_x - 1)/(c_s^2 drho), trained and run on the
// GPU.  Its prediction only initialises the populations; the lattice Boltzmann
// iteration then converges from there and removes its error (the paper's
// method is unchanged; the network is an accelerator of its steady state).
//
// Tensors are NHWC: activations bf16 with channel counts that are multiples
// of 16; weights [taps][Cout][Cin] bf16 with an FP32 master copy; FP32 bias.
// The convolution is an implicit GEMM on the tensor cores:
//   out[p, co] = act(b[co] + sum_{t, ci} in[p + off_t, ci] w[t][co][ci]),
// mma.sync m16n8k16 bf16 x bf16 -> fp32, operands staged in shared memory
// with cp.async (zero fill supplies the padding outside the image).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <string>

#include "lbm_launch.h"

namespace lbmgb {
namespace nn {

using bf16 = __nv_bfloat16;

namespace {

constexpr int kBM = 128;  // output pixels per block (one image row segment)
constexpr int kBN = 32;   // output channels per block
constexpr int kCK = 16;   // input channels per K step
constexpr int kPad = 8;   // bf16 padding per smem row (conflict-free 32-bit fragment loads)
constexpr int kRow = kCK + kPad;

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, bool valid) {
    const int n = valid ? 16 : 0;  // 0 source bytes: zero fill
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(g), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

}  // namespace

// grid: (ceil(W / 128), N * H, Cout / 32); block: 128 threads (4 warps x 32 pixels)
__global__ void __launch_bounds__(128)
    k_conv_fwd(const bf16* __restrict__ in, int N, int H, int W, int Cin, const bf16* __restrict__ w,
               const float* __restrict__ bias, int taps, int Cout, int relu, bf16* __restrict__ out,
               float* __restrict__ out_f32) {
    __shared__ __align__(16) bf16 patch[3][kBM + 2][kRow];
    __shared__ __align__(16) bf16 wsm[9][kBN][kRow];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tig = lane & 3;
    const int x0 = blockIdx.x * kBM;
    const int ny = blockIdx.y;  // n * H + y
    const int n = ny / H, y = ny % H;
    const int co0 = blockIdx.z * kBN;
    const int r0 = (taps == 9) ? 0 : 1, r1 = (taps == 9) ? 3 : 2;  // patch rows used
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

    for (int ci0 = 0; ci0 < Cin; ci0 += kCK) {
        // input patch rows y-1..y+1 (or y), columns x0-1 .. x0+128, channels ci0..ci0+15
        for (int i = tid; i < (r1 - r0) * (kBM + 2) * 2; i += 128) {
            const int half = i & 1, px = (i >> 1) % (kBM + 2), r = r0 + (i >> 1) / (kBM + 2);
            const int yy = y + r - 1, xx = x0 + px - 1;
            const bool ok = yy >= 0 && yy < H && xx >= 0 && xx < W;
            const bf16* src = ok ? in + (((size_t)n * H + yy) * W + xx) * Cin + ci0 + half * 8 : in;
            cp_async16((uint32_t)__cvta_generic_to_shared(&patch[r][px][half * 8]), src, ok);
        }
        for (int i = tid; i < taps * kBN * 2; i += 128) {
            const int half = i & 1, co = (i >> 1) % kBN, t = (i >> 1) / kBN;
            const bool ok = co0 + co < Cout;
            const bf16* src = ok ? w + ((size_t)t * Cout + co0 + co) * Cin + ci0 + half * 8 : w;
            cp_async16((uint32_t)__cvta_generic_to_shared(&wsm[t][co][half * 8]), src, ok);
        }
        cp_commit();
        cp_wait_all();
        __syncthreads();
        for (int t = 0; t < taps; ++t) {
            const int dy = (taps == 9) ? t / 3 : 1, dx = (taps == 9) ? t % 3 : 1;  // patch row, column shift
            uint32_t bfr[4][2];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                bfr[nt][0] = *reinterpret_cast<const uint32_t*>(&wsm[t][nt * 8 + g][2 * tig]);
                bfr[nt][1] = *reinterpret_cast<const uint32_t*>(&wsm[t][nt * 8 + g][2 * tig + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int p = warp * 32 + mt * 16 + g + dx;  // patch column of row g (x shift dx - 1)
                uint32_t afr[4];
                afr[0] = *reinterpret_cast<const uint32_t*>(&patch[dy][p][2 * tig]);
                afr[1] = *reinterpret_cast<const uint32_t*>(&patch[dy][p + 8][2 * tig]);
                afr[2] = *reinterpret_cast<const uint32_t*>(&patch[dy][p][2 * tig + 8]);
                afr[3] = *reinterpret_cast<const uint32_t*>(&patch[dy][p + 8][2 * tig + 8]);
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma16816(acc[mt][nt], afr, bfr[nt]);
            }
        }
        __syncthreads();
    }
    // epilogue: bias, activation, store bf16 pairs (and optionally fp32)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = x0 + warp * 32 + mt * 16 + g + h * 8;
                const int co = co0 + nt * 8 + 2 * tig;
                if (x >= W || co >= Cout) continue;
                float v0 = acc[mt][nt][2 * h] + (bias ? bias[co] : 0.f);
                float v1 = acc[mt][nt][2 * h + 1] + (bias ? bias[co + 1] : 0.f);
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                const size_t o = (((size_t)n * H + y) * W + x) * Cout + co;
                *reinterpret_cast<__nv_bfloat162*>(out + o) = __floats2bfloat162_rn(v0, v1);
                if (out_f32) {
                    out_f32[o] = v0;
                    out_f32[o + 1] = v1;
                }
            }
}

// Weights for the data gradient: wt[taps-1-t][ci][co] = w[t][co][ci] (the
// adjoint of a correlation is the correlation with flipped taps and swapped
// channel roles).
__global__ void k_wflip(const bf16* __restrict__ w, int taps, int Cout, int Cin, bf16* __restrict__ wt) {
    const size_t n = (size_t)taps * Cout * Cin;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ci = (int)(i % Cin);
        const int co = (int)((i / Cin) % Cout);
        const int t = (int)(i / ((size_t)Cin * Cout));
        wt[((size_t)(taps - 1 - t) * Cin + ci) * Cout + co] = w[i];
    }
}

// Weight and bias gradient, FP32 on the CUDA cores:
//   dw[t][co][ci] = sum_p g[p, co] in[p + off_t, ci],  db[co] = sum_p g[p, co].
// Block (x, ci tile, co tile) walks the 32-pixel row segments x, x + G, ...;
// each thread owns one (co, ci) pair and its taps.  Per-block partial sums go
// to `part` and k_wgrad_sum adds them in a fixed order (deterministic).
constexpr int kWP = 32;
__global__ void __launch_bounds__(256)
    k_wgrad_part(const bf16* __restrict__ in, const bf16* __restrict__ gout, int N, int H, int W, int Cin,
                 int Cout, int taps, float* __restrict__ part, float* __restrict__ bpart) {
    __shared__ float pin[3][kWP + 2][16];
    __shared__ float pg[kWP][16];
    const int tid = threadIdx.x;
    const int nseg = (W + kWP - 1) / kWP;
    const long total = (long)nseg * N * H;
    const int ci0 = blockIdx.y * 16, co0 = blockIdx.z * 16;
    const int co = tid / 16, ci = tid % 16;
    float a[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) a[t] = 0.f;
    float bsum = 0.f;
    for (long sidx = blockIdx.x; sidx < total; sidx += gridDim.x) {
        const int seg = (int)(sidx % nseg);
        const long ny = sidx / nseg;
        const int n = (int)(ny / H), y = (int)(ny % H), x0 = seg * kWP;
        __syncthreads();
        for (int i = tid; i < 3 * (kWP + 2) * 16; i += 256) {
            const int c = i % 16, px = (i / 16) % (kWP + 2), r = i / (16 * (kWP + 2));
            const int yy = y + r - 1, xx = x0 + px - 1;
            float v = 0.f;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = __bfloat162float(in[(((size_t)n * H + yy) * W + xx) * Cin + ci0 + c]);
            pin[r][px][c] = v;
        }
        for (int i = tid; i < kWP * 16; i += 256) {
            const int c = i % 16, px = i / 16;
            const int xx = x0 + px;
            pg[px][c] = xx < W ? __bfloat162float(gout[(((size_t)n * H + y) * W + xx) * Cout + co0 + c]) : 0.f;
        }
        __syncthreads();
        for (int px = 0; px < kWP; ++px) {
            const float gv = pg[px][co];
            bsum += gv;
            if (taps == 9) {
#pragma unroll
                for (int t = 0; t < 9; ++t) a[t] = fmaf(gv, pin[t / 3][px + t % 3][ci], a[t]);
            } else {
                a[0] = fmaf(gv, pin[1][px + 1][ci], a[0]);
            }
        }
    }
    const size_t blk = blockIdx.x;
    for (int t = 0; t < taps; ++t) part[((blk * taps + t) * Cout + co0 + co) * Cin + ci0 + ci] = a[t];
    if (blockIdx.y == 0 && ci == 0) bpart[blk * Cout + co0 + co] = bsum;
}

__global__ void k_wgrad_sum(const float* __restrict__ part, const float* __restrict__ bpart, int nblk, int taps,
                            int Cout, int Cin, float* __restrict__ dw, float* __restrict__ db, int accumulate) {
    const size_t nw = (size_t)taps * Cout * Cin;
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < nw) {
        float s = 0.f;
        for (int b = 0; b < nblk; ++b) s += part[(size_t)b * nw + i];
        dw[i] = accumulate ? dw[i] + s : s;
    }
    if (db && i < (size_t)Cout) {
        float s = 0.f;
        for (int b = 0; b < nblk; ++b) s += bpart[(size_t)b * Cout + i];
        db[i] = accumulate ? db[i] + s : s;
    }
}

// g_pre = g * (y > 0): gradient through a ReLU whose output is y.
__global__ void k_relu_bwd(const bf16* __restrict__ y, const bf16* __restrict__ gy, bf16* __restrict__ gx, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        gx[i] = __bfloat162float(y[i]) > 0.f ? gy[i] : __float2bfloat16(0.f);
}

// 2x2 average pooling (H, W even) and its adjoint.
__global__ void k_pool2_fwd(const bf16* __restrict__ in, int N, int H, int W, int C, bf16* __restrict__ out) {
    const int Ho = H / 2, Wo = W / 2;
    const size_t n = (size_t)N * Ho * Wo * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t p = i / C;
        const int x = (int)(p % Wo), y = (int)((p / Wo) % Ho), b = (int)(p / ((size_t)Wo * Ho));
        const size_t base = (((size_t)b * H + 2 * y) * W + 2 * x) * C + c;
        const float s = __bfloat162float(in[base]) + __bfloat162float(in[base + C]) +
                        __bfloat162float(in[base + (size_t)W * C]) + __bfloat162float(in[base + (size_t)W * C + C]);
        out[i] = __float2bfloat16(0.25f * s);
    }
}
__global__ void k_pool2_bwd(const bf16* __restrict__ gout, int N, int H, int W, int C, bf16* __restrict__ gin) {
    const size_t n = (size_t)N * H * W * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t p = i / C;
        const int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((size_t)W * H));
        const float g = __bfloat162float(gout[(((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]);
        gin[i] = __float2bfloat16(0.25f * g);
    }
}
// nearest-neighbour 2x upsampling (input H x W) and its adjoint
__global__ void k_up2_fwd(const bf16* __restrict__ in, int N, int H, int W, int C, bf16* __restrict__ out) {
    const size_t n = (size_t)N * 4 * H * W * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t p = i / C;
        const int x = (int)(p % (2 * W)), y = (int)((p / (2 * W)) % (2 * H)), b = (int)(p / ((size_t)4 * W * H));
        out[i] = in[(((size_t)b * H + y / 2) * W + x / 2) * C + c];
    }
}
__global__ void k_up2_bwd(const bf16* __restrict__ gout, int N, int H, int W, int C, bf16* __restrict__ gin) {
    const size_t n = (size_t)N * H * W * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t p = i / C;
        const int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((size_t)W * H));
        const size_t base = (((size_t)b * 2 * H + 2 * y) * 2 * W + 2 * x) * C + c;
        const size_t row = (size_t)2 * W * C;
        const float s = __bfloat162float(gout[base]) + __bfloat162float(gout[base + C]) +
                        __bfloat162float(gout[base + row]) + __bfloat162float(gout[base + row + C]);
        gin[i] = __float2bfloat16(s);
    }
}
// dst[p, dc0 + c] (+)= src[p, sc0 + c] for c < nc (concatenation and its adjoint)
__global__ void k_copy_ch(const bf16* __restrict__ src, int sld, int sc0, bf16* __restrict__ dst, int dld, int dc0,
                          int nc, size_t npix) {
    const size_t n = npix * nc;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % nc);
        const size_t p = i / nc;
        dst[p * dld + dc0 + c] = src[p * sld + sc0 + c];
    }
}

// Channel weights of the loss (at most 8 channels), passed by value.
struct ChanW {
    float w[8];
};

// Masked, channel-weighted mean squared error over fluid nodes and the first
// nout channels:
//   L = inv_count sum_{fluid p, c < nout} w_c (pred - target)^2,
//   grad = 2 w_c (pred - target) inv_count on fluid nodes, 0 elsewhere
//   (grad has the prediction's channel stride; padding channels get 0).
// Per-block partial losses, summed by k_sum_f32.
__global__ void __launch_bounds__(256)
    k_mse(const bf16* __restrict__ pred, int ld, const float* __restrict__ target, const uint8_t* __restrict__ solid,
          size_t npix, int nout, float inv_count, ChanW cw, bf16* __restrict__ grad, float* __restrict__ part) {
    __shared__ float sh[256];
    float acc = 0.f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < npix; p += (size_t)gridDim.x * blockDim.x) {
        const bool fl = solid[p] == 0;
        for (int c = 0; c < ld; ++c) {
            float gv = 0.f;
            if (c < nout && fl) {
                const float d = __bfloat162float(pred[p * ld + c]) - target[p * nout + c];
                acc += cw.w[c] * d * d;
                gv = 2.f * cw.w[c] * d * inv_count;
            }
            if (grad) grad[p * ld + c] = __float2bfloat16(gv);
        }
    }
    sh[threadIdx.x] = acc * inv_count;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_f32(const float* __restrict__ part, int n, float* __restrict__ out) {
    __shared__ float sh[256];
    float a = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) a += part[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// AdamW (Loshchilov & Hutter) on FP32 master weights, refreshing the bf16 copy.
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                        size_t n, float lr, float b1, float b2, float eps, float wd, float c1, float c2,
                        bf16* __restrict__ pb) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        const float pi = p[i] - lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16(pi);
    }
}

__global__ void k_add_bf16(const bf16* __restrict__ a, const bf16* __restrict__ b, bf16* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

// Network input of one sample: channel 0 = solid flag, 1 = x / (nx - 1),
// 2 = (tau - 1/2), channels 3..15 = 0.
__global__ void k_make_input(const uint8_t* __restrict__ solid, int H, int W, float tau_feat, bf16* __restrict__ out) {
    const size_t n = (size_t)H * W;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(p % W);
        bf16* o = out + p * 16;
        o[0] = __float2bfloat16(solid[p] ? 1.f : 0.f);
        o[1] = __float2bfloat16((float)x / (float)(W > 1 ? W - 1 : 1));
        o[2] = __float2bfloat16(tau_feat);
#pragma unroll
        for (int c = 3; c < 16; ++c) o[c] = __float2bfloat16(0.f);
    }
}

}  // namespace nn
}  // namespace lbmgb

// ---------------------------------------------------------------------------
// C ABI (device pointers; work enqueued on `stream`, nothing synchronised)
// ---------------------------------------------------------------------------
#include "lbm.h"

namespace {
using lbmgb::nn::bf16;

lbm_status nn_fail(const char* m) {
    lbmgb::set_thread_error(m);
    return LBM_ERR_ARG;
}
lbm_status nn_fail(const std::string& m, lbm_status s) {
    lbmgb::set_thread_error(m);
    return s;
}
// which tensor-core path the convolutions take (process-wide)
std::atomic<int> g_conv_impl{LBM_NN_CONV_AUTO};
// The automatic choice, from the measured times of the warm-start network's
// layers on GB300 (batch 8): tcgen05 is ahead only for wide layers on images of
// at least 64 pixels per row and 2048 pixels; shallow full-resolution layers and
// the small deep ones are faster with mma.sync.
bool use_tcgen05(int h, int w, int cin, int cout) {
    const int impl = g_conv_impl.load();
    if (impl != LBM_NN_CONV_AUTO) return impl == LBM_NN_CONV_TCGEN05;
    return cin >= 32 && cout >= 64 && w >= 64 && (long)h * w >= 2048;
}
lbm_status nn_launch_status() {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return LBM_OK;
    lbmgb::set_thread_error(std::string("kernel launch: ") + cudaGetErrorString(e));
    return LBM_ERR_CUDA;
}
bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
unsigned ew_grid(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b ? b : 1);
}
}  // namespace

extern "C" {

lbm_status lbm_nn_set_conv_impl(int32_t impl) {
    if (impl != LBM_NN_CONV_MMA_SYNC && impl != LBM_NN_CONV_TCGEN05 && impl != LBM_NN_CONV_AUTO)
        return nn_fail("unknown convolution path");
    g_conv_impl.store(impl);
    return LBM_OK;
}

int32_t lbm_nn_get_conv_impl(void) { return g_conv_impl.load(); }

lbm_status lbm_nn_sync_status(void* stream) {
    unsigned int word = 0;
    const cudaError_t e = lbmgb::nn::tc_error_take(&word, (cudaStream_t)stream);
    if (e != cudaSuccess) return nn_fail(std::string("lbm_nn_sync_status: ") + cudaGetErrorString(e), LBM_ERR_CUDA);
    if (word) return nn_fail("a tensor-core convolution gave up waiting for its MMAs (output incomplete)",
                             LBM_ERR_INTERNAL);
    return LBM_OK;
}

lbm_status lbm_nn_conv_fwd(const void* in, int32_t n, int32_t h, int32_t w, int32_t cin, const void* wts,
                           const float* bias, int32_t taps, int32_t cout, int32_t relu, void* out, float* out_f32,
                           void* stream) {
    if (!in || !wts || !out) return nn_fail("null tensor");
    if (n < 1 || h < 1 || w < 1 || cin < 16 || cin % 16 || cout < 16 || cout % 16 || (taps != 1 && taps != 9))
        return nn_fail("conv: need channels multiple of 16 and taps 1 or 9");
    if (!aligned16(in) || !aligned16(wts) || !aligned16(out)) return nn_fail("conv: tensors must be 16-byte aligned");
    if ((long)n * h > 65535) return nn_fail("conv: n*h must be <= 65535");
    if (use_tcgen05(h, w, cin, cout)) {
        const cudaError_t e = lbmgb::nn::launch_conv_fwd_tc(in, n, h, w, cin, wts, bias, taps, cout, relu, out,
                                                            out_f32, (cudaStream_t)stream);
        if (e != cudaSuccess) return nn_fail(std::string("conv (tcgen05) launch: ") + cudaGetErrorString(e), LBM_ERR_CUDA);
        return LBM_OK;
    }
    dim3 grid((w + lbmgb::nn::kBM - 1) / lbmgb::nn::kBM, n * h, (cout + lbmgb::nn::kBN - 1) / lbmgb::nn::kBN);
    lbmgb::nn::k_conv_fwd<<<grid, 128, 0, (cudaStream_t)stream>>>(
        (const bf16*)in, n, h, w, cin, (const bf16*)wts, bias, taps, cout, relu, (bf16*)out, out_f32);
    return nn_launch_status();
}

lbm_status lbm_nn_conv_bwd_data(const void* gout, int32_t n, int32_t h, int32_t w, int32_t cout, const void* wts,
                                int32_t taps, int32_t cin, void* wflip_scratch, void* gin, void* stream) {
    if (!gout || !wts || !wflip_scratch || !gin) return nn_fail("null tensor");
    if (cin % 16 || cout % 16 || cin < 16 || cout < 16 || (taps != 1 && taps != 9)) return nn_fail("conv bwd: bad shape");
    const size_t nw = (size_t)taps * cin * cout;
    lbmgb::nn::k_wflip<<<ew_grid(nw), 256, 0, (cudaStream_t)stream>>>((const bf16*)wts, taps, cout, cin,
                                                                      (bf16*)wflip_scratch);
    lbm_status s = nn_launch_status();
    if (s != LBM_OK) return s;
    return lbm_nn_conv_fwd(gout, n, h, w, cout, wflip_scratch, nullptr, taps, cin, 0, gin, nullptr, stream);
}

lbm_status lbm_nn_conv_bwd_weight(const void* in, const void* gout, int32_t n, int32_t h, int32_t w, int32_t cin,
                                  int32_t cout, int32_t taps, float* dw, float* db, int32_t accumulate, float* scratch,
                                  size_t scratch_floats, void* stream) {
    if (!in || !gout || !dw || !scratch) return nn_fail("null tensor");
    if (cin % 16 || cout % 16 || cin < 16 || cout < 16 || (taps != 1 && taps != 9)) return nn_fail("wgrad: bad shape");
    const size_t per = (size_t)taps * cout * cin + cout;
    const long nseg = (long)((w + lbmgb::nn::kWP - 1) / lbmgb::nn::kWP) * n * h;
    long G = (long)(scratch_floats / per);
    if (G < 1) return nn_fail("wgrad: scratch too small");
    if (G > nseg) G = nseg;
    if (G > 1024) G = 1024;
    float* part = scratch;
    float* bpart = scratch + (size_t)G * taps * cout * cin;
    dim3 grid((unsigned)G, cin / 16, cout / 16);
    lbmgb::nn::k_wgrad_part<<<grid, 256, 0, (cudaStream_t)stream>>>((const bf16*)in, (const bf16*)gout, n, h, w, cin,
                                                                   cout, taps, part, bpart);
    lbm_status s = nn_launch_status();
    if (s != LBM_OK) return s;
    const size_t nw = (size_t)taps * cout * cin;
    const size_t nt = nw > (size_t)cout ? nw : (size_t)cout;
    lbmgb::nn::k_wgrad_sum<<<(unsigned)((nt + 255) / 256), 256, 0, (cudaStream_t)stream>>>(part, bpart, (int)G, taps,
                                                                                          cout, cin, dw, db, accumulate);
    return nn_launch_status();
}

lbm_status lbm_nn_relu_bwd(const void* y, const void* gy, void* gx, size_t count, void* stream) {
    if (!y || !gy || !gx) return nn_fail("null tensor");
    lbmgb::nn::k_relu_bwd<<<ew_grid(count), 256, 0, (cudaStream_t)stream>>>((const bf16*)y, (const bf16*)gy,
                                                                            (bf16*)gx, count);
    return nn_launch_status();
}

lbm_status lbm_nn_pool2_fwd(const void* in, int32_t n, int32_t h, int32_t w, int32_t c, void* out, void* stream) {
    if (!in || !out || h % 2 || w % 2) return nn_fail("pool2: null tensor or odd size");
    lbmgb::nn::k_pool2_fwd<<<ew_grid((size_t)n * h * w * c / 4), 256, 0, (cudaStream_t)stream>>>((const bf16*)in, n, h,
                                                                                                w, c, (bf16*)out);
    return nn_launch_status();
}

lbm_status lbm_nn_pool2_bwd(const void* gout, int32_t n, int32_t h, int32_t w, int32_t c, void* gin, void* stream) {
    if (!gout || !gin || h % 2 || w % 2) return nn_fail("pool2: null tensor or odd size");
    lbmgb::nn::k_pool2_bwd<<<ew_grid((size_t)n * h * w * c), 256, 0, (cudaStream_t)stream>>>((const bf16*)gout, n, h, w,
                                                                                            c, (bf16*)gin);
    return nn_launch_status();
}

lbm_status lbm_nn_up2_fwd(const void* in, int32_t n, int32_t h, int32_t w, int32_t c, void* out, void* stream) {
    if (!in || !out) return nn_fail("up2: null tensor");
    lbmgb::nn::k_up2_fwd<<<ew_grid((size_t)n * 4 * h * w * c), 256, 0, (cudaStream_t)stream>>>((const bf16*)in, n, h, w,
                                                                                              c, (bf16*)out);
    return nn_launch_status();
}

lbm_status lbm_nn_up2_bwd(const void* gout, int32_t n, int32_t h, int32_t w, int32_t c, void* gin, void* stream) {
    if (!gout || !gin) return nn_fail("up2: null tensor");
    lbmgb::nn::k_up2_bwd<<<ew_grid((size_t)n * h * w * c), 256, 0, (cudaStream_t)stream>>>((const bf16*)gout, n, h, w, c,
                                                                                          (bf16*)gin);
    return nn_launch_status();
}

lbm_status lbm_nn_copy_channels(const void* src, int32_t sld, int32_t sc0, void* dst, int32_t dld, int32_t dc0,
                                int32_t nc, size_t npix, void* stream) {
    if (!src || !dst || nc < 1 || sc0 + nc > sld || dc0 + nc > dld) return nn_fail("copy_channels: bad arguments");
    lbmgb::nn::k_copy_ch<<<ew_grid(npix * nc), 256, 0, (cudaStream_t)stream>>>((const bf16*)src, sld, sc0, (bf16*)dst,
                                                                              dld, dc0, nc, npix);
    return nn_launch_status();
}

lbm_status lbm_nn_mse(const void* pred, int32_t ld, const float* target, const uint8_t* solid, size_t npix,
                      int32_t nout, const float* weights, float inv_count, void* grad, float* scratch256, float* loss,
                      void* stream) {
    if (!pred || !target || !solid || !scratch256 || !loss || nout < 1 || nout > ld || nout > 8)
        return nn_fail("mse: bad arguments");
    lbmgb::nn::ChanW cw;
    for (int c = 0; c < 8; ++c) cw.w[c] = (weights && c < nout) ? weights[c] : 1.f;
    lbmgb::nn::k_mse<<<256, 256, 0, (cudaStream_t)stream>>>((const bf16*)pred, ld, target, solid, npix, nout, inv_count,
                                                           cw, (bf16*)grad, scratch256);
    lbm_status s = nn_launch_status();
    if (s != LBM_OK) return s;
    lbmgb::nn::k_sum_f32<<<1, 256, 0, (cudaStream_t)stream>>>(scratch256, 256, loss);
    return nn_launch_status();
}

lbm_status lbm_nn_adamw(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps,
                        float wd, int32_t step, void* p_bf16, void* stream) {
    if (!p || !g || !m || !v || step < 1) return nn_fail("adamw: bad arguments");
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    lbmgb::nn::k_adamw<<<ew_grid(n), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, b1, b2, eps, wd, c1, c2,
                                                                     (bf16*)p_bf16);
    return nn_launch_status();
}

lbm_status lbm_nn_add(const void* a, const void* b, void* out, size_t n, void* stream) {
    if (!a || !b || !out) return nn_fail("null tensor");
    lbmgb::nn::k_add_bf16<<<ew_grid(n), 256, 0, (cudaStream_t)stream>>>((const bf16*)a, (const bf16*)b, (bf16*)out, n);
    return nn_launch_status();
}

lbm_status lbm_nn_f32_to_bf16(const float* a, void* b, size_t n, void* stream) {
    if (!a || !b) return nn_fail("null tensor");
    lbmgb::nn::k_f32_to_bf16<<<ew_grid(n), 256, 0, (cudaStream_t)stream>>>(a, (bf16*)b, n);
    return nn_launch_status();
}

lbm_status lbm_nn_make_input(const uint8_t* solid, int32_t h, int32_t w, float tau_feat, void* out, void* stream) {
    if (!solid || !out || h < 1 || w < 1) return nn_fail("make_input: bad arguments");
    lbmgb::nn::k_make_input<<<ew_grid((size_t)h * w), 256, 0, (cudaStream_t)stream>>>(solid, h, w, tau_feat, (bf16*)out);
    return nn_launch_status();
}

}  // extern "C"
