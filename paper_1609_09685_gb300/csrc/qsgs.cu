// qsgs.cu -- QSGS porous-mask generation on the GPU (Sec. 2's "randomly
// generated quartet structure", generated by the quartet structure generation
// set of Wang et al. 2007, growing the solid phase).
//
// Draws come from a counter-based splitmix64 hash (Steele, Lea & Flood 2014):
// the stream key of iteration t is output t+1 of splitmix64(seed), and the draw
// for (cell, neighbour slot) is the high 32 bits of output cell*32 + slot + 1 of
// splitmix64(key).  Every decision is an integer comparison of a draw against
// floor(p 2^32), and the partial last iteration keeps the candidates with the
// smallest (draw, cell) keys, so the mask depends only on (seed, sizes,
// probabilities, porosity) and not on launch geometry or timing.
#include <cuda_runtime.h>

#include <cmath>

#include "lbm_launch.h"

namespace lbmgb {

namespace {

constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ull;
constexpr uint64_t kNoKey = ~0ull;

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// n-th output (n >= 1) of splitmix64 seeded with `s`.
__host__ __device__ __forceinline__ uint64_t sm_out(uint64_t s, uint64_t n) { return sm_mix(s + kGamma * n); }

__device__ __forceinline__ uint32_t draw(uint64_t key, uint64_t cell, uint32_t slot) {
    return (uint32_t)(sm_out(key, cell * 32ull + slot + 1ull) >> 32);
}

struct Slots {
    int nd;
    int8_t dx[26], dy[26], dz[26];
    uint32_t thr[26];
};

__device__ __forceinline__ void add_count(unsigned long long* counter, bool hit) {
    const unsigned b = __ballot_sync(0xffffffffu, hit);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(counter, (unsigned long long)__popc(b));
}

__global__ void k_cores(uint64_t key, uint64_t n, uint32_t thr, uint64_t* __restrict__ keys,
                        unsigned long long* __restrict__ counter) {
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c = base + threadIdx.x;
        bool hit = false;
        if (c < n) {
            const uint32_t h = draw(key, c, 0u);
            hit = h < thr;
            keys[c] = hit ? (((uint64_t)h << 32) | c) : kNoKey;
        }
        add_count(counter, hit);
    }
}

__global__ void k_grow(uint64_t key, int nx, int ny, int nz, Slots S, const uint8_t* __restrict__ start,
                       uint64_t* __restrict__ keys, unsigned long long* __restrict__ counter) {
    const uint64_t n = (uint64_t)nx * ny * nz;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c = base + threadIdx.x;
        bool hit = false;
        if (c < n) {
            uint64_t best = kNoKey;
            if (!start[c]) {
                const int x = (int)(c % (uint64_t)nx);
                const int y = (int)((c / (uint64_t)nx) % (uint64_t)ny);
                const int z = (int)(c / ((uint64_t)nx * ny));
                for (int d = 0; d < S.nd; ++d) {
                    const int X = x + S.dx[d], Y = y + S.dy[d], Z = z + S.dz[d];
                    if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) continue;
                    if (!start[((uint64_t)Z * ny + Y) * nx + X]) continue;
                    const uint32_t h = draw(key, c, (uint32_t)d);
                    if (h < S.thr[d]) {
                        const uint64_t k = ((uint64_t)h << 32) | c;
                        best = k < best ? k : best;
                    }
                }
            }
            hit = best != kNoKey;
            keys[c] = best;
        }
        add_count(counter, hit);
    }
}

__global__ void k_count_below(const uint64_t* __restrict__ keys, uint64_t n, uint64_t T,
                              unsigned long long* __restrict__ counter) {
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c = base + threadIdx.x;
        add_count(counter, c < n && keys[c] < T);
    }
}

__global__ void k_apply(const uint64_t* __restrict__ keys, uint64_t n, uint64_t T, uint8_t* __restrict__ solid) {
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (uint64_t)gridDim.x * blockDim.x)
        if (keys[c] < T) solid[c] = 1;
}

uint32_t prob_thr(double p) {
    if (!(p > 0.0)) return 0u;
    const double t = std::floor(p * 4294967296.0);
    return t >= 4294967295.0 ? 4294967295u : (uint32_t)t;
}

unsigned grid_for(uint64_t n) {
    uint64_t b = (n + 255) / 256;
    if (b > 152ull * 16) b = 152ull * 16;
    return (unsigned)(b ? b : 1);
}

}  // namespace

int qsgs_generate(uint64_t seed, int nx, int ny, int nz, double core_p, double porosity, double d_face,
                  uint8_t* d_mask, const QsgsScratch& sc, cudaStream_t st, int* iterations,
                  cudaError_t* cuda_err) {
    *cuda_err = cudaSuccess;
    if (nx < 1 || ny < 1 || nz < 1 || !(porosity >= 0.0 && porosity <= 1.0)) return -1;
    const uint64_t N = (uint64_t)nx * ny * nz;
    const uint64_t S = (uint64_t)std::floor((1.0 - porosity) * (double)N + 0.5);
    Slots sl{};
    const uint32_t tf = prob_thr(d_face), te = prob_thr(d_face / 2.0), tc = prob_thr(d_face / 4.0);
    for (int dz = (nz > 1 ? -1 : 0); dz <= (nz > 1 ? 1 : 0); ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int k = (dx != 0) + (dy != 0) + (dz != 0);
                if (k == 0) continue;
                sl.dx[sl.nd] = (int8_t)dx;
                sl.dy[sl.nd] = (int8_t)dy;
                sl.dz[sl.nd] = (int8_t)dz;
                sl.thr[sl.nd] = k == 1 ? tf : (k == 2 ? (nz > 1 ? te : tc) : tc);
                ++sl.nd;
            }

#define QCK(x)                       \
    do {                             \
        cudaError_t e_ = (x);        \
        if (e_ != cudaSuccess) {     \
            *cuda_err = e_;          \
            return -2;               \
        }                            \
    } while (0)

    auto read_counter = [&](unsigned long long* out) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(sc.host_counter, sc.counter, sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        *out = *sc.host_counter;
        return e;
    };
    // Make candidates solid: all if they fit under S, else the (S - count)
    // smallest keys, found by bisection on the key value (keys are unique).
    auto accept = [&](uint64_t ncand, uint64_t& count) -> cudaError_t {
        if (ncand == 0) return cudaSuccess;
        uint64_t T = kNoKey;
        if (count + ncand > S) {
            const uint64_t need = S - count;
            uint64_t lo = 0, hi = kNoKey;  // count(<lo) < need <= count(<hi)
            while (hi - lo > 1) {
                const uint64_t mid = lo + (hi - lo) / 2;
                cudaError_t e = cudaMemsetAsync(sc.counter, 0, sizeof(unsigned long long), st);
                if (e != cudaSuccess) return e;
                k_count_below<<<grid_for(N), 256, 0, st>>>(sc.keys, N, mid, sc.counter);
                unsigned long long c = 0;
                e = read_counter(&c);
                if (e != cudaSuccess) return e;
                if (c >= need) hi = mid;
                else lo = mid;
            }
            T = hi;
            count = S;
        } else {
            count += ncand;
        }
        k_apply<<<grid_for(N), 256, 0, st>>>(sc.keys, N, T, d_mask);
        return cudaGetLastError();
    };

    QCK(cudaMemsetAsync(d_mask, 0, N, st));
    uint64_t count = 0;
    unsigned long long nc = 0;
    QCK(cudaMemsetAsync(sc.counter, 0, sizeof(unsigned long long), st));
    k_cores<<<grid_for(N), 256, 0, st>>>(sm_out(seed, 1), N, prob_thr(core_p), sc.keys, sc.counter);
    QCK(cudaGetLastError());
    QCK(read_counter(&nc));
    QCK(accept(nc, count));
    int t = 0;
    while (count < S) {
        if (count == 0) return -3;
        ++t;
        if (t > kMaxGrowthIterations) return -4;
        QCK(cudaMemcpyAsync(sc.start, d_mask, N, cudaMemcpyDeviceToDevice, st));
        QCK(cudaMemsetAsync(sc.counter, 0, sizeof(unsigned long long), st));
        k_grow<<<grid_for(N), 256, 0, st>>>(sm_out(seed, (uint64_t)t + 1), nx, ny, nz, sl, sc.start, sc.keys,
                                            sc.counter);
        QCK(cudaGetLastError());
        QCK(read_counter(&nc));
        QCK(accept(nc, count));
    }
    QCK(cudaStreamSynchronize(st));
#undef QCK
    if (iterations) *iterations = t;
    return 0;
}

}  // namespace lbmgb
