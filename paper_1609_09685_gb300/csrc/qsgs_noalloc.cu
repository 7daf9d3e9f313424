// qsgs_noalloc.cu -- QSGS mask generation into a caller-owned device buffer
// without any allocation.
//
// Some callers cannot allocate GPU memory while they run: a host that has
// handed its whole device budget to its own pool allocator, code running under
// a memory policy that forbids cudaMalloc / cudaFree between set-up and
// shutdown, or an embedding that must never trigger the implicit device
// synchronisation cudaFree can cause.  lbm_qsgs_noalloc serves them: the
// scratch QSGS needs (one 64-bit draw key and one start-of-iteration byte per
// cell, plus a candidate counter) lives in the file-scope array below, sized
// for at most kNoAllocMaxCells cells.  Every GPU that loads the library holds
// this array (about 9 MB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lbm.h"
#include "lbm_launch.h"

namespace {

constexpr uint64_t kNoAllocMaxCells = 1ull << 20;  // 1,048,576 cells (e.g. 1200 x 600 fits)
constexpr size_t kKeysBytes = kNoAllocMaxCells * sizeof(uint64_t);
constexpr size_t kStartBytes = kNoAllocMaxCells;
constexpr size_t kScratchBytes = kKeysBytes + kStartBytes + 256;

// keys | start mask | counter, each 256-byte aligned
static __device__ __align__(256) unsigned char g_qsgs_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

thread_local unsigned long long t_host_counter;  // pageable readback slot, one per host thread

lbm_status noalloc_fail(lbm_status s, const std::string& m) {
    lbmgb::set_thread_error(m);  // reported by lbm_last_error(NULL)
    return s;
}

}  // namespace

extern "C" {

lbm_status lbm_qsgs_noalloc(uint64_t seed, int32_t nx, int32_t ny, int32_t nz, double core_p, double porosity,
                            double d_face, void* stream, uint8_t* mask_dev_out, int32_t* iterations) {
    if (!mask_dev_out) return noalloc_fail(LBM_ERR_ARG, "mask_dev_out is null");
    if (nx < 1 || ny < 1 || nz < 1) return noalloc_fail(LBM_ERR_ARG, "sizes must be >= 1");
    const uint64_t N = (uint64_t)nx * ny * nz;
    if (N > kNoAllocMaxCells)
        return noalloc_fail(LBM_ERR_ARG, "nx*ny*nz = " + std::to_string(N) +
                                             " exceeds the allocation-free scratch limit of " +
                                             std::to_string(kNoAllocMaxCells) + " cells");
    if (!(porosity >= 0.0 && porosity <= 1.0)) return noalloc_fail(LBM_ERR_ARG, "porosity outside [0,1]");
    if (!(core_p >= 0.0 && core_p <= 1.0) || !(d_face >= 0.0 && d_face <= 1.0))
        return noalloc_fail(LBM_ERR_ARG, "probabilities outside [0,1]");

    // Once per device, with that device current: the device address of the
    // scratch array (its name in host code is only a host-side stand-in).
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LBM_ERR_INTERNAL, "device ordinal beyond 64");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_qsgs_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_scratch_addr[dev];
    }
    lbmgb::QsgsScratch sc{};
    sc.keys = reinterpret_cast<uint64_t*>(base);
    sc.start = base + kKeysBytes;
    sc.counter = reinterpret_cast<unsigned long long*>(base + kKeysBytes + kStartBytes);
    sc.host_counter = &t_host_counter;
    int it = 0;
    cudaError_t ce = cudaSuccess;
    // qsgs_generate writes every key and start byte it reads and zeroes the
    // counter before each count, so leftovers of an earlier call never leak in.
    const int r = lbmgb::qsgs_generate(seed, nx, ny, nz, core_p, porosity, d_face, mask_dev_out, sc,
                                       (cudaStream_t)stream, &it, &ce);
    if (r == -2) return noalloc_fail(LBM_ERR_CUDA, std::string("qsgs kernels: ") + cudaGetErrorString(ce));
    if (r == -1) return noalloc_fail(LBM_ERR_ARG, "bad qsgs arguments");
    if (r == -3) return noalloc_fail(LBM_ERR_INTERNAL, "no solid core to grow from");
    if (r == -4) return noalloc_fail(LBM_ERR_INTERNAL, "growth iteration cap reached before the target porosity");
    if (iterations) *iterations = it;
    return LBM_OK;
}

}  // extern "C"
