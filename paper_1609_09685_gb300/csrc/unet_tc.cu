// unet_tc.cu -- the warm-start network's 3x3 / 1x1 convolution on the 5th
// generation tensor cores (tcgen05, sm_103a): an implicit GEMM
//   out[p, co] = act(b[co] + sum_{t, ci} in[p + off_t, ci] w[t][co][ci])
// with the accumulator in tensor memory.
//
// A block computes M = 128 output pixels (a segment of one image row) x NT <= 128
// output channels.  The K loop runs over 16-channel chunks; per chunk the
// block stages, with cp.async (zero fill outside the image), the three input
// rows y-1..y+1 over pixels x0-1 .. x0+128 and the taps' weights for its
// channels, into one of two shared-memory stages.  Operands use the canonical
// K-major layout without swizzle: a core matrix is 8 rows x 16 bytes (8 bf16
// channels), rows 16 bytes apart, the next 8 rows 128 bytes further (SBO) and
// the other 8 channels of the chunk LBO bytes away.  A tap's A operand is the
// staged row dy read from pixel dx on: since pixel rows are uniformly 16 bytes
// apart, the shift is a 16 * dx byte offset of the descriptor, so one staged
// patch feeds all nine taps without copies.  One thread issues the nine
// tcgen05.mma (kind::f16, bf16 x bf16 -> fp32, M = 128, N = NT, K = 16) of a
// chunk and tcgen05.commit signals an mbarrier when they have read the stage,
// which then takes the chunk after next.  The epilogue reads the accumulator
// with tcgen05.ld (warp w owns tensor-memory lanes 32 w .. 32 w + 31, i.e.
// pixels), adds the bias, applies the ReLU and stores bf16 (and optionally
// fp32) NHWC.
//
// Every wait is bounded: a wait that gives up sets the file's device error
// flag (read by lbm_nn_sync_status), the block frees its tensor memory and
// leaves without storing.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "lbm_launch.h"

namespace lbmgb {
namespace nn {

using bf16 = __nv_bfloat16;

__device__ unsigned int g_tc_error;  // nonzero once a tensor-core convolution's wait gave up

namespace {

constexpr int kM = 128;         // output pixels per block
constexpr int kNmax = 128;      // output channels per block (at most)
constexpr int kPx = kM + 2;     // staged pixels per row (x0 - 1 .. x0 + 128)
constexpr int kAHalf = kPx * 16;  // bytes of one 8-channel half of a staged row
constexpr int kARow = 2 * kAHalf;
constexpr int kWaitTries = 1 << 22;

// Shared memory of a block whose channel tile is nt: two stages of the staged
// input rows and the taps' weights, then two mbarriers and the tensor-memory
// address.  Sized by nt, so that shallow layers fit more blocks per SM.
template <int TAPS>
struct TcGeo {
    static constexpr int ROWS = TAPS == 9 ? 3 : 1;
    static constexpr int A_BYTES = ROWS * kARow;
    __host__ __device__ static constexpr int stage(int nt) { return A_BYTES + TAPS * 2 * nt * 16; }
    __host__ __device__ static constexpr int smem(int nt) { return 2 * stage(nt) + 32; }
};
static_assert(TcGeo<9>::A_BYTES % 16 == 0 && TcGeo<9>::stage(16) % 16 == 0, "16-byte aligned operands");

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K) and
// stride (M/N) byte offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = n, M = 128.
__device__ __forceinline__ uint32_t instr_desc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    for (int i = 0; i < kWaitTries; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace

// grid: (ceil(W / 128), N * H, ceil(Cout / 128)); block: 128 threads
template <int TAPS>
__global__ void __launch_bounds__(128)
    k_conv_fwd_tc(const bf16* __restrict__ in, int N, int H, int W, int Cin, const bf16* __restrict__ w,
                  const float* __restrict__ bias, int Cout, int relu, bf16* __restrict__ out,
                  float* __restrict__ out_f32) {
    using G = TcGeo<TAPS>;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * kM;
    const int n = blockIdx.y / H, y = blockIdx.y % H;
    const int co0 = blockIdx.z * kNmax;
    const int NT = min(kNmax, Cout - co0);  // a multiple of 16
    const int STAGE = G::stage(NT);
    const uint32_t bars = saddr(sm + 2 * STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * STAGE + 16);
    const uint32_t ncols = NT <= 32 ? 32u : (NT <= 64 ? 64u : 128u);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bars + 8u * s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = instr_desc(NT);
    const int chunks = Cin / 16;
    bool ok = true;
    for (int c = 0; c < chunks && ok; ++c) {
        const int s = c & 1;
        // the stage is free once the MMAs of chunk c - 2 have read it
        if (c >= 2) ok = bar_wait(bars + 8u * s, ((c >> 1) - 1) & 1);
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        unsigned char* st = sm + s * STAGE;
        const uint32_t a0 = saddr(st), b0 = a0 + G::A_BYTES;
        const int ci0 = c * 16;
        for (int i = tid; i < G::ROWS * 2 * kPx; i += 128) {
            const int px = i % kPx, kh = (i / kPx) & 1, r = i / (2 * kPx);
            const int yy = y + (TAPS == 9 ? r - 1 : 0), xx = x0 + px - 1;
            const bool v = yy >= 0 && yy < H && xx >= 0 && xx < W;
            const bf16* src = v ? in + (((size_t)n * H + yy) * W + xx) * Cin + ci0 + kh * 8 : in;
            cp16(a0 + (uint32_t)((r * 2 + kh) * kAHalf + px * 16), src, v);
        }
        for (int i = tid; i < TAPS * 2 * NT; i += 128) {
            const int co = i % NT, kh = (i / NT) & 1, t = i / (2 * NT);
            const bf16* src = w + ((size_t)t * Cout + co0 + co) * Cin + ci0 + kh * 8;
            cp16(b0 + (uint32_t)(((t * 2 + kh) * NT + co) * 16), src, true);
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        // the tensor cores read shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int t = 0; t < TAPS; ++t) {
                const int dy = TAPS == 9 ? t / 3 : 0, dx = TAPS == 9 ? t % 3 : 1;
                const uint64_t da = smem_desc(a0 + (uint32_t)(dy * kARow + dx * 16), kAHalf, 128);
                const uint64_t db = smem_desc(b0 + (uint32_t)(t * 2 * NT * 16), (uint32_t)NT * 16u, 128);
                mma(tmem, da, db, idesc, (c > 0 || t > 0) ? 1u : 0u);
            }
            commit(bars + 8u * s);
        }
    }
    // all MMAs done: the last chunk's commit completes after every earlier one
    if (ok) {
        const int cl = chunks - 1;
        ok = bar_wait(bars + 8u * (cl & 1), (cl >> 1) & 1);
    }
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(&g_tc_error, 1u);
        // give MMAs still in flight one more bounded wait before the memory goes
        if (chunks > 0) bar_wait(bars + 8u * ((chunks - 1) & 1), ((chunks - 1) >> 1) & 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int m = warp * 32 + lane;
        const int x = x0 + m;
        const size_t o = (((size_t)n * H + y) * W + x) * Cout + co0;
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (x < W) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = __uint_as_float(r[j]) + (bias ? bias[co0 + c0 + j] : 0.f);
                    if (relu) v[j] = fmaxf(v[j], 0.f);
                }
                uint4 pk[2];
                uint32_t* pw = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                    pw[j] = *reinterpret_cast<const uint32_t*>(&h2);
                }
                uint4* dst = reinterpret_cast<uint4*>(out + o + c0);
                dst[0] = pk[0];
                dst[1] = pk[1];
                if (out_f32) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) out_f32[o + c0 + j] = v[j];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

cudaError_t launch_conv_fwd_tc(const void* in, int N, int H, int W, int Cin, const void* w, const float* bias,
                               int taps, int Cout, int relu, void* out, float* out_f32, cudaStream_t st) {
    const dim3 grid((W + kM - 1) / kM, N * H, (Cout + kNmax - 1) / kNmax);
    const int nt = Cout < kNmax ? Cout : kNmax;  // the widest channel tile of the launch
    if (taps == 9) {
        static std::atomic<uint64_t> set9{0};  // bit d: attribute set on device d
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        const uint64_t bit = 1ull << (dev & 63);
        if (dev >= 64 || !(set9.load() & bit)) {
            e = cudaFuncSetAttribute(k_conv_fwd_tc<9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     TcGeo<9>::smem(kNmax));
            if (e != cudaSuccess) return e;
            if (dev < 64) set9.fetch_or(bit);
        }
        k_conv_fwd_tc<9><<<grid, 128, TcGeo<9>::smem(nt), st>>>((const bf16*)in, N, H, W, Cin, (const bf16*)w, bias,
                                                            Cout, relu, (bf16*)out, out_f32);
    } else {
        k_conv_fwd_tc<1><<<grid, 128, TcGeo<1>::smem(nt), st>>>((const bf16*)in, N, H, W, Cin, (const bf16*)w, bias,
                                                            Cout, relu, (bf16*)out, out_f32);
    }
    return cudaGetLastError();
}

cudaError_t tc_error_take(unsigned int* word, cudaStream_t st) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyFromSymbol(word, g_tc_error, sizeof(unsigned int));
    if (e != cudaSuccess) return e;
    const unsigned int zero = 0;
    return cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(unsigned int));
}

}  // namespace nn
}  // namespace lbmgb
