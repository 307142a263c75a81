// pgg_kernels_direct.cu -- one sublattice step in place on a bit-packed lattice, operands
// read straight from global memory (L1/L2), no shared-memory staging.
//
// A step only writes the sites of one sublattice, which are at least 4 apart, and an
// update reads only the Manhattan ball of radius 3 around its site (Section IV, Fig. 3;
// radius 2 for the pairwise game of Section VI, which loads 5 rows instead of 7),
// so the step can run in place with every thread reading its neighbourhood directly: the
// only words another thread writes during the step are words of the same sublattice row,
// and the bits it changes there are never among the bits this thread uses.
//
// Thread task: one sublattice row a and UPT consecutive 32-column words of it (8 UPT
// sites). The thread keeps the 7 rows x 3 words around the current word in registers and
// slides right one word per unit; the direction draws of the task come from one Philox call
// (64 sites per call, so UPT = 8 needs one call and UPT = 4 half of one). The cooperator
// count is kept as a running total: each step adds the change it made.
#include <cuda_runtime.h>

#include "pgg_device.cuh"
#include "pgg_internal.h"
#include "pgg_unit.cuh"

// Minimum resident CTAs per SM requested from the register allocator.
#ifndef PGG_DIRECT_MIN_BLOCKS
#define PGG_DIRECT_MIN_BLOCKS 1
#endif

namespace pgg {
namespace {

struct DirectParams {
    uint32_t *lat;  // bit-packed lattice, L rows of Lw words, updated in place
    int L, Lw;
    uint64_t k;     // sublattice step index
    uint64_t seed;
    int tasks_per_row;     // Lw / UPT
    uint32_t task_magic;   // ceil(2^32 / tasks_per_row), 0 when tasks_per_row == 1
    int n_tasks;           // (L / 4) * tasks_per_row
    const uint32_t *table;
    unsigned long long *running;  // cooperator count, += this step's change (nullable)
    int *status;                  // | 4 when an index check fails (checked build)
    PhiloxKeys rk;
};

template <int UPT, int OJ, int GAME>
__device__ __forceinline__ long long direct_body(const DirectParams &p, const PhiloxKeys &rk,
                                                 const uint32_t *__restrict__ s_table, int oi) {
    long long delta = 0;
    const uint32_t kl = static_cast<uint32_t>(p.k), kh = static_cast<uint32_t>(p.k >> 32) | kTagDir;
    const int stride = gridDim.x * blockDim.x;
    const long long n_words = static_cast<long long>(p.L) * p.Lw;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < p.n_tasks; t += stride) {
        const int a = p.task_magic ? static_cast<int>(__umulhi(static_cast<uint32_t>(t), p.task_magic)) : t;
        const int w0 = (t - a * p.tasks_per_row) * UPT;
        const int i = 4 * a + oi;
        // word offsets of rows i-3 .. i+3 (periodic)
        int rowoff[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) rowoff[q] = wrap_small(i - 3 + q, p.L) * p.Lw;
        const int wprev = w0 == 0 ? p.Lw - 1 : w0 - 1;
        // rows the game reads (the pairwise game reads two lines less, Section VI)
        uint32_t wl[7], wc[7], wr[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            wl[q] = reads_row<GAME>(q) && index_ok(rowoff[q] + wprev, n_words, p.status) ? p.lat[rowoff[q] + wprev] : 0u;
            wc[q] = reads_row<GAME>(q) && index_ok(rowoff[q] + w0, n_words, p.status) ? p.lat[rowoff[q] + w0] : 0u;
        }
        const uint4 dcall = philox_rk(make_uint4(static_cast<uint32_t>(w0 >> 3), static_cast<uint32_t>(a), kl, kh), rk);
        UnitCtx u;
        u.k = p.k;
        u.a = static_cast<uint32_t>(a);
        u.msk = kNib;
        // kept rolled: one copy of the unit body keeps the hot code inside the instruction cache
#pragma unroll 1
        for (int s = 0; s < UPT; ++s) {
            const int w = w0 + s;
            const int wn = w + 1 == p.Lw ? 0 : w + 1;
#pragma unroll
            for (int q = 0; q < 7; ++q)
                wr[q] = reads_row<GAME>(q) && index_ok(rowoff[q] + wn, n_words, p.status) ? p.lat[rowoff[q] + wn] : 0u;
            u.gw = w;
            u.d16 = (word_of(dcall, (w >> 1) & 3) >> (16 * (w & 1))) & 0xFFFFu;
            uint32_t sx;
            const uint32_t flips = game_flips<OJ, GAME>(wl, wc, wr, u, rk, s_table, sx);
            if (flips && index_ok(rowoff[3] + w, n_words, p.status)) {
                p.lat[rowoff[3] + w] = wc[3] ^ (flips << OJ);
                delta += __popc(flips & ~sx) - __popc(flips & sx);
            }
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                wl[q] = wc[q];
                wc[q] = wr[q];
            }
        }
    }
    return delta;
}

template <int UPT, int BLOCK, int GAME>
__global__ void __launch_bounds__(BLOCK, PGG_DIRECT_MIN_BLOCKS) k_step_direct(const __grid_constant__ DirectParams p) {
    constexpr int kEntries = GAME == kPairGame ? kPairEntries : kTableEntries;
    __shared__ uint32_t s_table[kEntries];
    __shared__ int s_off;
    __shared__ long long s_warp[BLOCK / 32];
    for (int t = threadIdx.x; t < kEntries; t += blockDim.x) s_table[t] = p.table[t];
    if (threadIdx.x == 0) s_off = draw_offset(p.seed, p.k);
    __syncthreads();
    const PhiloxKeys rk = p.rk;
    const int o = s_off;
    long long delta;
    switch (o & 3) {
        case 0: delta = direct_body<UPT, 0, GAME>(p, rk, s_table, o >> 2); break;
        case 1: delta = direct_body<UPT, 1, GAME>(p, rk, s_table, o >> 2); break;
        case 2: delta = direct_body<UPT, 2, GAME>(p, rk, s_table, o >> 2); break;
        default: delta = direct_body<UPT, 3, GAME>(p, rk, s_table, o >> 2); break;
    }
    if (p.running) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) delta += __shfl_down_sync(0xffffffffu, delta, s);
        if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = delta;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long b = 0;
            for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) b += s_warp[w];
            if (b) atomicAdd(p.running, static_cast<unsigned long long>(b));
        }
    }
}

template <int UPT, int BLOCK, int GAME>
int resident_grid() {
    static int grid = 0;  // per instance and process; the library drives one device type
    if (!grid) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_direct<UPT, BLOCK, GAME>, BLOCK, 0) != cudaSuccess)
            return 0;
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    return grid;
}

template <int UPT, int BLOCK, int GAME>
cudaError_t launch_direct_instance(const DirectParams &p, cudaStream_t s) {
    const int grid = resident_grid<UPT, BLOCK, GAME>();
    if (!grid) return cudaErrorUnknown;
    const int need = (p.n_tasks + BLOCK - 1) / BLOCK;
    k_step_direct<UPT, BLOCK, GAME><<<need < grid ? need : grid, BLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

template <int GAME>
cudaError_t launch_direct_game(const DirectParams &p, int upt, int block, cudaStream_t s) {
    // small blocks spread the step's few tasks evenly over the SMs
    if (block == 128)
        return upt == 4 ? launch_direct_instance<4, 128, GAME>(p, s) : launch_direct_instance<8, 128, GAME>(p, s);
    if (block == 256)
        return upt == 4 ? launch_direct_instance<4, 256, GAME>(p, s) : launch_direct_instance<8, 256, GAME>(p, s);
    return upt == 4 ? launch_direct_instance<4, 64, GAME>(p, s) : launch_direct_instance<8, 64, GAME>(p, s);
}

}  // namespace

bool direct_supported(int layout, int L) { return layout == kPacked && L >= 256 && L % 256 == 0; }

cudaError_t launch_step_direct(int game, uint32_t *lat, int L, uint64_t seed, uint64_t k, const uint32_t *table,
                               unsigned long long *running, int *status, int upt, int block, cudaStream_t s) {
    if (L < 256 || L % 256 != 0 || (upt != 4 && upt != 8)) return cudaErrorInvalidValue;
    DirectParams p;
    p.lat = lat;
    p.L = L;
    p.Lw = L / 32;
    p.k = k;
    p.seed = seed;
    p.tasks_per_row = p.Lw / upt;
    p.task_magic = p.tasks_per_row <= 1 ? 0u
                                        : static_cast<uint32_t>((0x100000000ull + p.tasks_per_row - 1) / p.tasks_per_row);
    p.n_tasks = (L / 4) * p.tasks_per_row;
    p.table = table;
    p.running = running;
    p.status = status;
    p.rk = philox_round_keys(seed);
    return game == kPairGame ? launch_direct_game<kPairGame>(p, upt, block, s)
                             : launch_direct_game<kGroupGame>(p, upt, block, s);
}

}  // namespace pgg
