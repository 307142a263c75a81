// pgg_kernels_tiled.cu -- shared-memory tiled, temporally blocked sublattice-step kernel.
//
// One CTA owns a tile of tile_y x tile_x sites. It stages the tile plus a halo in shared
// memory as bit rows (one bit per site, for both lattice layouts), applies `steps`
// consecutive sublattice steps there, and writes the interior back. An update reads the
// Manhattan ball of radius R = 3 around its site (Section IV, Fig. 3: the halo is
// three rows deep; R = 2 for the pairwise game, one line less, Section VI), so after step j
// (0-based) of k only the sites within R (k - 1 - j) of the interior are still needed and
// still correct; the halo is therefore R k sites wide and the updated region shrinks by R
// per step. Every random draw is keyed by global (step, site), so the
// halo copies that several tiles compute redundantly agree bit for bit.
//
// Work unit: one 32-column word of one sublattice row. Its 8 sublattice sites sit at bits
// oj + 4m (m = 0..7), four bits apart, so after shifting the word's neighbourhood by oj
// every quantity of the 8 sites lives in one nibble of a 32-bit register:
//   Y(di, dj)    bit 4m = strategy of the site at (i + di, j_m + dj)
//   n(di, dj)    = Y(di,dj) + Y(di,dj-1) + Y(di,dj+1) + Y(di-1,dj) + Y(di+1,dj)
//                  the cooperator count of the group centred at (i+di, j_m+dj) (Fig. 1)
//   S(z)         = n(z) + n(z's 4 neighbours), kept as two partial nibble sums (<= 15, <= 10)
// S(x) and S(y) (y chosen by the direction draw) index the threshold table of Eq. (3).
#include <cuda_runtime.h>

#include "pgg_device.cuh"
#include "pgg_internal.h"
#include "pgg_unit.cuh"

namespace pgg {
namespace {

constexpr int kMaxSteps = 16;
constexpr size_t kMaxSmem = 227 * 1024 - 1024;  // leave room for static shared memory

struct TiledParams {
    const void *src;
    void *dst;
    int L, Lw;  // lattice side, 32-site words per row
    uint64_t seed, k0;
    int steps;
    int tile_x, tile_y;
    int tiles_x, tiles_y;
    int R;          // read radius of the game's update (3 groups, 2 pairwise)
    int H, hw;      // halo in sites (R steps) and in words
    int RP;         // shared-memory column pitch in words (odd, >= tile rows + 2H)
    int dir_slot;   // uint32 words of one step's direction buffer
    int dir_words;  // uint32 words reserved for the two direction buffers
    const uint32_t *table;
    unsigned long long *count_out;
    int *status;           // | 4 when an index check fails (checked build); nullable
    long long tile_words;  // words of the shared tile buffer (Wr * RP for a full tile)
    PhiloxKeys rk;  // round keys of the seed
};

__host__ __device__ constexpr int halo_words(int steps, int R) { return (R * (steps - 1) + 31) / 32 + 1; }

// 32 bytes of 0/1 -> 32 bits (byte n -> bit n).
__device__ __forceinline__ uint32_t nibble_of_bytes(uint32_t x) { return ((x * 0x00204081u) >> 21) & 0xFu; }

__device__ __forceinline__ uint32_t pack32(const uint4 lo, const uint4 hi) {
    return nibble_of_bytes(lo.x) | nibble_of_bytes(lo.y) << 4 | nibble_of_bytes(lo.z) << 8 |
           nibble_of_bytes(lo.w) << 12 | nibble_of_bytes(hi.x) << 16 | nibble_of_bytes(hi.y) << 20 |
           nibble_of_bytes(hi.z) << 24 | nibble_of_bytes(hi.w) << 28;
}

__device__ __forceinline__ uint32_t bytes_of_nibble(uint32_t nib) {
    return (nib & 1u) | ((nib >> 1) & 1u) << 8 | ((nib >> 2) & 1u) << 16 | ((nib >> 3) & 1u) << 24;
}

// Exact quotient t / d for t, d < 2^16 with m = ceil(2^32 / d); d = 1 (where m would be
// 2^32) is encoded as m = 0.
__host__ __device__ __forceinline__ uint32_t div_magic(uint32_t d) {
    return d <= 1 ? 0u : static_cast<uint32_t>((0x100000000ull + d - 1) / d);
}
__device__ __forceinline__ int div_by_magic(int t, uint32_t m) {
    return m == 0u ? t : static_cast<int>(__umulhi(static_cast<uint32_t>(t), m));
}

// The part of the tile one fused step updates: sublattice rows r_first, r_first + 4, ...
// below row_hi, and local words [w_lo, w_hi) (sites outside [col_lo, col_hi) masked).
// Direction words are grouped by call-aligned runs of 8 global words, runs c_lo .. c_lo +
// n_runs - 1 in unwrapped global word coordinates U = x0w - hw + w.
struct StepGeom {
    int row_hi, col_lo, col_hi, w_lo, w_hi, r_first, n_srows, n_words, c_lo, n_runs;
};

__device__ __forceinline__ StepGeom step_geom(const TiledParams &p, int x0w, int ih, int iw, int j, int oi) {
    StepGeom g;
    const int e = p.R * (p.steps - 1 - j);
    const int row_lo = p.H - e;
    g.row_hi = p.H + ih + e;
    g.col_lo = 32 * p.hw - e;
    g.col_hi = 32 * p.hw + iw + e;
    g.w_lo = g.col_lo >> 5;
    g.w_hi = (g.col_hi + 31) >> 5;
    g.r_first = row_lo + ((oi + p.H - row_lo) & 3);
    g.n_srows = g.r_first < g.row_hi ? (g.row_hi - g.r_first + 3) >> 2 : 0;
    g.n_words = g.w_hi - g.w_lo;
    g.c_lo = (x0w - p.hw + g.w_lo) >> 3;
    g.n_runs = ((x0w - p.hw + g.w_hi - 1) >> 3) - g.c_lo + 1;
    return g;
}

// Direction codes of step j for every unit of its region: one Philox call per sublattice
// row and run of 8 global words (64 sites), stored as its four words at
// s_dir[srow * 4 n_runs + 4 (run - c_lo) + i]; word i holds the 16-bit codes of global
// words 8 run + 2i (low half) and 8 run + 2i + 1 (high half).
__device__ __forceinline__ void tile_dirs(const TiledParams &p, const PhiloxKeys &rk, uint32_t *s_dir,
                                          int y0, int x0w, int ih, int iw, int j, int oi, int tid,
                                          int nthreads) {
    const StepGeom g = step_geom(p, x0w, ih, iw, j, oi);
    const uint64_t k = p.k0 + j;
    const uint32_t kl = static_cast<uint32_t>(k), kh = static_cast<uint32_t>(k >> 32) | kTagDir;
    const int n_tasks = g.n_srows * g.n_runs;
    const uint32_t magic = div_magic(static_cast<uint32_t>(g.n_runs));
    const bool aligned = (p.Lw & 7) == 0;  // every run lies in one call
    for (int t = tid; t < n_tasks; t += nthreads) {
        const int sr = div_by_magic(t, magic);
        const int c = g.c_lo + (t - sr * g.n_runs);
        const int r = g.r_first + 4 * sr;
        const uint32_t a = static_cast<uint32_t>(wrap_small(y0 - p.H + r, p.L) >> 2);
        uint4 out;
        if (aligned) {
            const int dg = wrap_small(8 * c, p.Lw) >> 3;
            out = philox_rk(make_uint4(static_cast<uint32_t>(dg), a, kl, kh), rk);
        } else {
            // the run crosses the periodic edge of a lattice whose width is not a multiple
            // of 8 words: take each word's codes from its own call
            uint32_t w4[4] = {0u, 0u, 0u, 0u};
            int cached = -1;
            uint4 call = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int gw = wrap_small(8 * c + i, p.Lw);
                if ((gw >> 3) != cached) {
                    cached = gw >> 3;
                    call = philox_rk(make_uint4(static_cast<uint32_t>(cached), a, kl, kh), rk);
                }
                const uint32_t d16 = (word_of(call, (gw >> 1) & 3) >> (16 * (gw & 1))) & 0xFFFFu;
                w4[i >> 1] |= d16 << (16 * (i & 1));
            }
            out = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
        reinterpret_cast<uint4 *>(s_dir)[sr * g.n_runs + (c - g.c_lo)] = out;
    }
}

// One sublattice step over the update region of the tile, for column offset OJ. The tile
// is column-major in shared memory: word (row r, word w) at s_tile[w * RP + r].
template <int LAYOUT, int BLOCK, int OJ, int GAME>
__device__ __forceinline__ void tile_step(const TiledParams &p, const PhiloxKeys &rk, uint32_t *s_tile,
                                          const uint32_t *__restrict__ s_table,
                                          const uint32_t *__restrict__ s_dir, int y0, int x0w,
                                          int ih, int iw, int j, int oi) {
    const uint64_t k = p.k0 + j;
    const StepGeom g = step_geom(p, x0w, ih, iw, j, oi);
    const int n_tasks = g.n_srows * g.n_words;
    const uint32_t magic = div_magic(static_cast<uint32_t>(g.n_words));
    const bool in_place = (p.steps == 1);
    const int RP = p.RP;

    for (int t = threadIdx.x; t < n_tasks; t += BLOCK) {
        const int sr = div_by_magic(t, magic);
        const int w = g.w_lo + (t - sr * g.n_words);
        const int r = g.r_first + 4 * sr;
        uint32_t *col = s_tile + w * RP + r;
        const long long ci = static_cast<long long>(w) * RP + r;  // index of col[0] in the tile
        uint32_t wl[7], wc[7], wr[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            // rows r-3 .. r+3; a game reads only rows r-R .. r+R, all inside the staged tile
            const bool rq = reads_row<GAME>(q);
            wl[q] = rq && index_ok(ci + q - 3 - RP, p.tile_words, p.status) ? col[q - 3 - RP] : 0u;
            wc[q] = rq && index_ok(ci + q - 3, p.tile_words, p.status) ? col[q - 3] : 0u;
            wr[q] = rq && index_ok(ci + q - 3 + RP, p.tile_words, p.status) ? col[q - 3 + RP] : 0u;
        }
        const int U = x0w - p.hw + w;
        const int grow = wrap_small(y0 - p.H + r, p.L);
        UnitCtx u;
        u.k = k;
        u.a = static_cast<uint32_t>(grow >> 2);
        u.gw = wrap_small(U, p.Lw);
        u.d16 = (s_dir[sr * 4 * g.n_runs + 4 * ((U >> 3) - g.c_lo) + ((U >> 1) & 3)] >> (16 * (U & 1))) & 0xFFFFu;
        u.msk = kNib;
        if (w == g.w_lo || w == g.w_hi - 1) {
            // sites at local columns 32 w + OJ + 4 m inside [col_lo, col_hi)
            const int base = 32 * w + OJ;
            u.msk = nibble_range((g.col_lo - base + 3) >> 2, (g.col_hi - base + 3) >> 2);
        }
        uint32_t sx;
        const uint32_t flips = game_flips<OJ, GAME>(wl, wc, wr, u, rk, s_table, sx);
        if (flips && index_ok(ci, p.tile_words, p.status)) {
            const uint32_t nw = wc[3] ^ (flips << OJ);
            col[0] = nw;
            if (in_place) {
                if (LAYOUT == kPacked) {
                    if (index_ok(static_cast<long long>(grow) * p.Lw + u.gw, static_cast<long long>(p.L) * p.Lw, p.status))
                        static_cast<uint32_t *>(p.dst)[static_cast<size_t>(grow) * p.Lw + u.gw] = nw;
                } else {
                    uint8_t *rowp = static_cast<uint8_t *>(p.dst) + static_cast<size_t>(grow) * p.L + 32 * u.gw + OJ;
                    const uint32_t newbits = (sx ^ flips);
#pragma unroll
                    for (int m = 0; m < 8; ++m)
                        if ((flips & (1u << (4 * m))) &&
                            index_ok(static_cast<long long>(grow) * p.L + 32 * u.gw + OJ + 4 * m, static_cast<long long>(p.L) * p.L, p.status))
                            rowp[4 * m] = static_cast<uint8_t>((newbits >> (4 * m)) & 1u);
                }
            }
        }
    }
}

// Minimum resident CTAs per SM requested from the register allocator.
#ifndef PGG_TILED_MIN_BLOCKS
#define PGG_TILED_MIN_BLOCKS 1
#endif

template <int LAYOUT, int BLOCK, int GAME>
__global__ void __launch_bounds__(BLOCK, PGG_TILED_MIN_BLOCKS) k_step_tiled(const __grid_constant__ TiledParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *s_table = smem;
    int *s_off = reinterpret_cast<int *>(smem + kTableEntries);
    uint32_t *s_dir = smem + kTableEntries + kMaxSteps;
    uint32_t *s_tile = smem + kTableEntries + kMaxSteps + p.dir_words;
    __shared__ unsigned long long s_warp_count[BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = BLOCK / 32;
    const PhiloxKeys rk = p.rk;
    const int RP = p.RP;

    constexpr int kEntries = GAME == kPairGame ? kPairEntries : kTableEntries;
    for (int t = threadIdx.x; t < kEntries; t += BLOCK) s_table[t] = p.table[t];
    if (threadIdx.x < p.steps) s_off[threadIdx.x] = draw_offset(p.seed, p.k0 + threadIdx.x);

    const int n_tiles = p.tiles_x * p.tiles_y;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int ty = tile / p.tiles_x;
        const int tx = tile - ty * p.tiles_x;
        const int y0 = ty * p.tile_y, x0 = tx * p.tile_x;
        const int ih = min(p.tile_y, p.L - y0), iw = min(p.tile_x, p.L - x0);
        const int x0w = x0 >> 5;
        const int n_rows = ih + 2 * p.H;
        const int Wr = (iw >> 5) + 2 * p.hw;
        __syncthreads();  // offsets ready; the previous tile is fully consumed
        // stage tile + halo as bit rows, column-major
        for (int r = warp; r < n_rows; r += kWarps) {
            const int grow = wrap_small(y0 - p.H + r, p.L);
            int gw = wrap_small(x0w - p.hw + lane, p.Lw);
            for (int w = lane; w < Wr; w += 32) {
                uint32_t bits;
                if (LAYOUT == kPacked) {
                    bits = static_cast<const uint32_t *>(p.src)[static_cast<size_t>(grow) * p.Lw + gw];
                } else {
                    const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const uint8_t *>(p.src) +
                                                                       static_cast<size_t>(grow) * p.L + 32 * gw);
                    bits = pack32(src[0], src[1]);
                }
                if (index_ok(static_cast<long long>(w) * RP + r, p.tile_words, p.status)) s_tile[w * RP + r] = bits;
                gw = wrap_small(gw + 32, p.Lw);
            }
        }
        tile_dirs(p, rk, s_dir, y0, x0w, ih, iw, 0, s_off[0] >> 2, threadIdx.x, BLOCK);
        __syncthreads();
        for (int j = 0; j < p.steps; ++j) {
            const int o = s_off[j];
            const int oi = o >> 2;
            const uint32_t *dir_j = s_dir + (j & 1) * p.dir_slot;
            switch (o & 3) {
                case 0: tile_step<LAYOUT, BLOCK, 0, GAME>(p, rk, s_tile, s_table, dir_j, y0, x0w, ih, iw, j, oi); break;
                case 1: tile_step<LAYOUT, BLOCK, 1, GAME>(p, rk, s_tile, s_table, dir_j, y0, x0w, ih, iw, j, oi); break;
                case 2: tile_step<LAYOUT, BLOCK, 2, GAME>(p, rk, s_tile, s_table, dir_j, y0, x0w, ih, iw, j, oi); break;
                default: tile_step<LAYOUT, BLOCK, 3, GAME>(p, rk, s_tile, s_table, dir_j, y0, x0w, ih, iw, j, oi); break;
            }
            if (j + 1 < p.steps)
                tile_dirs(p, rk, s_dir + ((j + 1) & 1) * p.dir_slot, y0, x0w, ih, iw, j + 1,
                          s_off[j + 1] >> 2, threadIdx.x, BLOCK);
            __syncthreads();
        }
        // write the interior back (fused launches) and count it
        unsigned long long cnt = 0;
        const int iwords = iw >> 5;
        for (int rr = warp; rr < ih; rr += kWarps) {
            for (int ww = lane; ww < iwords; ww += 32) {
                const long long ti = static_cast<long long>(p.hw + ww) * RP + p.H + rr;
                const uint32_t bits = index_ok(ti, p.tile_words, p.status) ? s_tile[ti] : 0u;
                cnt += __popc(bits);
                if (p.steps > 1) {
                    const int grow = y0 + rr;
                    const int gw = x0w + ww;
                    // the word's 32 sites, as one packed word or 32 bytes
                    if (!index_ok(static_cast<long long>(grow) * p.Lw + gw, static_cast<long long>(p.L) * p.Lw, p.status)) {
                    } else if (LAYOUT == kPacked) {
                        static_cast<uint32_t *>(p.dst)[static_cast<size_t>(grow) * p.Lw + gw] = bits;
                    } else {
                        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint8_t *>(p.dst) +
                                                               static_cast<size_t>(grow) * p.L + 32 * gw);
                        dst[0] = make_uint4(bytes_of_nibble(bits), bytes_of_nibble(bits >> 4),
                                            bytes_of_nibble(bits >> 8), bytes_of_nibble(bits >> 12));
                        dst[1] = make_uint4(bytes_of_nibble(bits >> 16), bytes_of_nibble(bits >> 20),
                                            bytes_of_nibble(bits >> 24), bytes_of_nibble(bits >> 28));
                    }
                }
            }
        }
        if (p.count_out) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
            if (lane == 0) s_warp_count[warp] = cnt;
            __syncthreads();
            if (threadIdx.x < 32) {
                cnt = threadIdx.x < kWarps ? s_warp_count[threadIdx.x] : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
                if (threadIdx.x == 0 && cnt) atomicAdd(p.count_out, cnt);
            }
        }
    }
}

// Largest region of one step: sublattice rows and call-aligned runs (direction buffer).
void dir_slot_dims(int steps, int R, int tile_x, int tile_y, int *srows, int *runs) {
    const int e = R * (steps - 1);
    *srows = (tile_y + 2 * e + 3) / 4 + 1;
    *runs = (tile_x + 2 * e + 31) / 32 / 8 + 3;
}

int column_pitch(int steps, int R, int tile_y) {
    const int rows = tile_y + 2 * R * steps;
    return (rows & 1) ? rows : rows + 1;
}

size_t smem_bytes_for(int steps, int R, int tile_x, int tile_y, int *dir_slot, int *dir_words) {
    const int hw = halo_words(steps, R);
    const int Wr = tile_x / 32 + 2 * hw;
    int sr, runs;
    dir_slot_dims(steps, R, tile_x, tile_y, &sr, &runs);
    const int slot = 4 * sr * runs;  // uint32 words per step
    if (dir_slot) *dir_slot = slot;
    if (dir_words) *dir_words = 2 * slot;
    return sizeof(uint32_t) * (static_cast<size_t>(kTableEntries) + kMaxSteps + 2 * static_cast<size_t>(slot) +
                               static_cast<size_t>(Wr) * column_pitch(steps, R, tile_y));
}

template <int LAYOUT, int GAME>
cudaError_t launch_instance(const TiledParams &p, size_t smem, int grid, cudaStream_t s) {
    constexpr int kBlock = 256;
    auto kernel = k_step_tiled<LAYOUT, kBlock, GAME>;
    // the opt-in limit covers static plus dynamic shared memory; raise the dynamic
    // limit of this instance only as far as a launch needs
    static size_t configured = 48 * 1024;
    if (smem > configured) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
        if (e != cudaSuccess) return e;
        if (smem + fa.sharedSizeBytes > static_cast<size_t>(optin)) return cudaErrorInvalidValue;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    kernel<<<grid, kBlock, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

int read_radius(int game) { return game == kPairGame ? kReadRadius<kPairGame> : kReadRadius<kGroupGame>; }

size_t tiled_smem_bytes(int layout, int game, int steps, int tile_x, int tile_y) {
    (void)layout;
    if (steps < 1 || steps > kMaxSteps || tile_x < 64 || tile_x % 64 || tile_y < 4 || tile_y % 4) return 0;
    const size_t b = smem_bytes_for(steps, read_radius(game), tile_x, tile_y, nullptr, nullptr);
    return b <= kMaxSmem ? b : 0;
}

cudaError_t launch_step_tiled(const TiledArgs &a, cudaStream_t s) {
    if (a.L < 64 || a.L % 64 || a.tile_x % 64 || a.tile_y % 4 || a.tile_x > a.L || a.tile_y > a.L)
        return cudaErrorInvalidValue;
    if (a.steps < 1 || a.steps > kMaxSteps) return cudaErrorInvalidValue;
    if (a.steps > 1 && a.src == a.dst) return cudaErrorInvalidValue;
    TiledParams p;
    p.src = a.src;
    p.dst = a.dst;
    p.L = a.L;
    p.Lw = a.L / 32;
    p.seed = a.seed;
    p.k0 = a.k0;
    p.steps = a.steps;
    p.tile_x = a.tile_x;
    p.tile_y = a.tile_y;
    p.tiles_x = (a.L + a.tile_x - 1) / a.tile_x;
    p.tiles_y = (a.L + a.tile_y - 1) / a.tile_y;
    p.R = read_radius(a.game);
    p.H = p.R * a.steps;
    p.hw = halo_words(a.steps, p.R);
    p.RP = column_pitch(a.steps, p.R, a.tile_y);
    p.table = a.table;
    p.count_out = a.count_out;
    p.status = a.status;
    p.tile_words = static_cast<long long>(a.tile_x / 32 + 2 * p.hw) * p.RP;
    p.rk = philox_round_keys(a.seed);
    const size_t smem = smem_bytes_for(a.steps, p.R, a.tile_x, a.tile_y, &p.dir_slot, &p.dir_words);
    if (smem > kMaxSmem) return cudaErrorInvalidValue;
    const int grid = p.tiles_x * p.tiles_y;
    if (a.game == kPairGame)
        return a.layout == kPacked ? launch_instance<kPacked, kPairGame>(p, smem, grid, s)
                                   : launch_instance<kU8, kPairGame>(p, smem, grid, s);
    return a.layout == kPacked ? launch_instance<kPacked, kGroupGame>(p, smem, grid, s)
                               : launch_instance<kU8, kGroupGame>(p, smem, grid, s);
}

}  // namespace pgg
