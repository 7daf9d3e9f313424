// lbm_device.cuh -- device-side types and lattice traits of the GB300 LBM
// library (shared by the library's own .cu files only).
#pragma once
#include <cstddef>
#include <cstdint>

namespace lbmgb {

constexpr int kNumObs = 8;  // per-domain observables, see lbm.h lbm_step_observe
constexpr int kSegW = 32;   // nodes per segment (one warp lane per node)

// Velocity sets of Qian, d'Humieres & Lallemand (1992), in the order that
// include/lbm.h documents.  Components are looked up with compile-time
// indices after loop unrolling, so every table access folds to a constant.
struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    static constexpr int NROW = 3;  // neighbour rows (dy in -1..1)
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
        return t[i][a];
    }
    __host__ __device__ static constexpr double wd(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    static constexpr int NROW = 9;  // neighbour rows (dy, dz in -1..1)
    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int t[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},   {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return t[i][a];
    }
    __host__ __device__ static constexpr double wd(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// Direction with velocity (x, y, z); -1 when absent.
template <class L>
__host__ __device__ constexpr int find_dir(int x, int y, int z) {
    for (int j = 0; j < L::Q; ++j)
        if (L::c(j, 0) == x && L::c(j, 1) == y && L::c(j, 2) == z) return j;
    return -1;
}
template <class L>
__host__ __device__ constexpr int opp(int i) {
    return find_dir<L>(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
}
// Direction i with its y (and/or z) component reversed: specular reflection.
template <class L>
__host__ __device__ constexpr int flip(int i, bool fy, bool fz) {
    return find_dir<L>(L::c(i, 0), fy ? -L::c(i, 1) : L::c(i, 1), fz ? -L::c(i, 2) : L::c(i, 2));
}

// One domain of a batch as the kernels see it (16-byte aligned: the staged
// gather step copies a domain's record with a bulk copy).
struct alignas(16) DomainDev {
    int32_t nx, ny, nz;  // nz = 1 in 2D
    int32_t nseg;        // segments per x-row, ceil(nx / 32)
    uint32_t seg_base;   // first global segment of the domain
    uint32_t nseg_dom;   // nseg * ny * nz
    float omega;         // 1 / tau (BGK; the even-part rate of TRT)
    float omega_m;       // odd-part rate of TRT, 1 / tau_minus; equals omega for BGK
    float drho_in;       // rho_in - rho_0 (outlet carries rho_0 exactly)
    float rho0;          // rho_0 = rho_out
    int32_t active;      // 0 once retired by the steady-state control
    uint64_t mask_base;  // byte offset of the domain's dense mask
    uint32_t item_base;  // first strip work item of the domain
    uint32_t nitems;     // strip work items of the domain
    uint32_t fluid_begin;  // compact index of the domain's first fluid node (a multiple of 32)
    uint32_t fluid_end;    // one past its last fluid node
    // x-slab of a larger domain (lbm_slab_create); plain domains: x0 = 0,
    // nx_glob = nx, ghost = 0.  A ghost column (bit 0: x = 0, bit 1:
    // x = nx - 1) holds the neighbouring slab's populations: it is pulled
    // from but never written and never observed.
    int32_t x0;       // global x of column 0
    int32_t nx_glob;  // global N_x (the initial density ramp and Kn use it)
    uint32_t ghost;
};
static_assert(sizeof(DomainDev) == 96, "DomainDev is 96 bytes");

// Neighbour window of one segment, read by the stream-collide kernel:
//   x = lo | hi << 32 holds 34 fluid bits, bit k <-> node x = 32 s - 1 + k
//   (the left neighbour's last node, the segment's 32 nodes, the right
//   neighbour's first node); z = compact index of node 32 s - 1 if that node is
//   fluid, else of the segment's first fluid node (offset - left bit);
//   w = the segment's own mask.
using SegWindow = uint4;

// Strip work item: up to 255 consecutive rows y0 .. y0 + nrows - 1 (one z
// plane) at segment column s of one domain.
//   x = global segment of (s, y0, z); y = domain | nrows << 24;
//   z = y0 | z << 16;                  w = s.
using StripItem = uint4;

// Tile of the staged gather step: up to kTileRowsMax rows (y0 .. y0 + nrows - 1)
// of one z plane at nsegs <= kTileSegs consecutive segment columns s0 .. of one
// domain, with the compact range of every source row it pulls from.  Source
// row q (0 .. nrows + 1) of plane zq is row y0 - 1 + q clamped onto the domain
// (a clamped row stands for the mirror image at a specular face); its range
// [a0, a0 + 4 n16) covers the compact slots of nodes x = 32 s0 - 1 ..
// 32 (s0 + nsegs), widened to 16-byte boundaries (n16 = 0: no fluid there).
// Index of (plane zq, row q): zq * 6 + q, zq = 0 (z - 1), 1 (z), 2 (z + 1); 2D
// tiles use zq = 0 only.
constexpr int kTileSegs = 4;
constexpr int kTileRowsMax = 4;
struct GatherTile {
    uint32_t dom;
    uint32_t yz;     // y0 | z << 16
    uint32_t shape;  // nrows | nsegs << 8 | s0 << 16
    uint32_t dims;   // ny | nseg << 16 of the domain
    uint32_t a0[18];
    uint16_t n16[18];
    uint32_t wbase;  // window record of (plane z, row 0, segment s0)
};
static_assert(sizeof(GatherTile) == 128, "GatherTile is 128 bytes");

// Band of the band gather step (D2Q9): up to kBandSegs consecutive segment
// columns s0 .. s0 + nsegs - 1 of one domain and up to kBandRowsMax rows
// y0 .. y0 + nrows - 1, walked top to bottom by one block.
//   x = domain; y = y0 | nrows << 16; z = s0 | nsegs << 16;
//   w = index of the band's first range record.
// Range records (one per row y0 - 1 .. y0 + nrows, rows outside the domain
// included): x = first compact index of the row's staged range, a multiple of
// 4; y = its length in 16-byte units (0: nothing to stage).  The range covers
// the compact slots of nodes x = 32 s0 - 1 .. 32 (s0 + nsegs) of the row.
using BandItem = uint4;
constexpr int kBandSegs = 8;
constexpr int kBandRowsMax = 64;
// Rows per band when lbm_options.band_rows is 0 (0: the direct gather step).
constexpr int kBandRowsDefault = 0;
// L2-blocked pairs: MB of populations per block when lbm_options.pair_block_mb
// is 0 (0: unblocked pairs), and the largest block size accepted.
constexpr int kPairBlockMbDefault = 0;
constexpr int kPairBlockMbMax = 4096;
// Fused pair work units: strips per gather unit, local items per local unit,
// and how far (MB of blocks) the gather step runs ahead of the local step.
constexpr uint32_t kFusedGather = 4;
constexpr uint32_t kFusedLocal = 16;
#ifndef LBM_FUSED_LAG_MB
#define LBM_FUSED_LAG_MB 32
#endif
constexpr int kFusedLagMb = LBM_FUSED_LAG_MB;

// Arguments of the hot stream-collide kernel.
struct HotArgs {
    const DomainDev* dom;
    const SegWindow* win;
    const StripItem* items;
    uint32_t nitems;
    uint32_t pstride;        // elements between direction planes (Q * pstride < 2^32)
    const float* src[19];    // direction planes of the state being read
    float* dst[19];          // direction planes of the state being written
    const uint2* vitems;     // local-step work items: (first compact index, domain), one warp each
    uint32_t nvitems;
    const uint32_t* face;    // 2 bits per compact slot: bit 0 inlet (x = 0), bit 1 outlet (x = N_x - 1)
    const GatherTile* tiles; // staged gather step: tile list
    uint32_t ntiles;
    uint32_t* err;           // device error word (bit 0: a staged copy never completed)
    const BandItem* bands;   // band gather step: band list
    uint32_t nbands;
    const uint2* band_rng;   // band gather step: range records
};

// Work queue of the fused in-place pair (k_aa_pair_fused).
struct PairFused {
    const uint4* units;      // x = kind (0 gather, 1 local) | block << 1; y = first item; z = item count
    uint32_t nunits;
    uint32_t nblocks;
    const uint32_t* total;   // gather units of each block
    uint32_t* ctr;           // [0] next ticket, [1] unused, [2 + k] gather units of block k done;
                             // zeroed before every launch
};

// Arguments shared by every segment kernel.
struct Geometry {
    const DomainDev* dom;
    const uint32_t* seg_dom;   // domain of each global segment
    const uint32_t* seg_mask;  // fluid bits of each segment (bit l = node x = 32 s + l)
    const uint32_t* seg_off;   // compact index of the segment's first fluid node
    uint32_t nseg_total;
    uint64_t pstride;  // elements between direction planes of a population array
};

}  // namespace lbmgb
