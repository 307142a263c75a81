// pgg_kernels_tiled.cu -- shared-memory tiled, temporally blocked sublattice-step kernel.
//
// One CTA owns a tile of tile_y x tile_x sites. It stages the tile plus a halo in shared
// memory as bit rows (one bit per site, for both lattice layouts), applies `steps`
// consecutive sublattice steps there, and writes the interior back. An update reads the
// Manhattan ball of radius 3 around its site (Section IV, Fig. 3: "three lines outward"),
// so after step j (0-based) of k only the sites within 3 (k - 1 - j) of the interior are
// still needed and still correct; the halo is therefore 3k sites wide and the updated
// region shrinks by 3 per step. Every random draw is keyed by global (step, site), so the
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

namespace pgg {
namespace {

constexpr uint32_t kNib = 0x11111111u;
constexpr uint32_t kLowNib = 0x0F0F0F0Fu;
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
    int H, hw;     // halo in sites (3 steps) and in words
    int pitch;     // physical words per shared-memory row
    int dir_slot;  // uint16 entries of one step's direction buffer
    int dir_words; // uint32 words reserved for the two direction buffers
    const uint32_t *table;
    unsigned long long *count_out;
};

__host__ __device__ constexpr int halo_words(int steps) { return (3 * (steps - 1) + 31) / 32 + 1; }

template <int WPT>
__host__ __device__ constexpr int skew(int w) { return w + w / WPT; }

__device__ __forceinline__ int mod_pos(int v, int m) {
    v %= m;
    return v < 0 ? v + m : v;
}

// The 32 columns starting D columns to the right (D < 0: left) of the word whose left,
// centre and right neighbours are l, c, r.
template <int D>
__device__ __forceinline__ uint32_t window(uint32_t l, uint32_t c, uint32_t r) {
    static_assert(D >= -6 && D <= 6, "window shift out of range");
    if constexpr (D == 0) return c;
    else if constexpr (D > 0) return __funnelshift_r(c, r, D);
    else return __funnelshift_l(l, c, -D);
}

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

__device__ __forceinline__ uint32_t mux(uint32_t sel, uint32_t if0, uint32_t if1) {
    return (if0 & ~sel) | (if1 & sel);
}

// Sites m in [m_lo, m_hi) as nibble bits.
__device__ __forceinline__ uint32_t nibble_range(int m_lo, int m_hi) {
    m_lo = max(m_lo, 0);
    m_hi = min(m_hi, 8);
    if (m_hi <= m_lo) return 0u;
    const uint32_t hi = m_hi == 8 ? kNib : (kNib & ((1u << (4 * m_hi)) - 1u));
    const uint32_t lo = kNib & ~((1u << (4 * m_lo)) - 1u);
    return hi & lo;
}

struct UnitCtx {
    uint64_t seed, k;
    uint32_t a;       // sublattice row index of the unit
    int gw;           // global word index of the unit
    uint32_t d16;     // direction codes of the 8 sites (2 bits each)
    uint32_t msk;     // sites of the unit inside the update region (nibble bits)
};

// One unit: returns the flip mask (nibble bits) of its 8 sites. Rows q = 0..6 of wl/wc/wr
// are the unit's row offsets -3..+3.
template <int OJ>
__device__ __forceinline__ uint32_t unit_flips(const uint32_t (&wl)[7], const uint32_t (&wc)[7],
                                               const uint32_t (&wr)[7], const UnitCtx &u,
                                               const uint32_t *__restrict__ s_table, uint32_t &sx_out) {
#define PGG_Y(DI, DJ) (window<(DJ) + OJ>(wl[(DI) + 3], wc[(DI) + 3], wr[(DI) + 3]) & kNib)
    // direction codes of site m into nibble m (bits 4m, 4m+1)
    uint32_t d = u.d16;
    d = (d | (d << 8)) & 0x00FF00FFu;
    d = (d | (d << 4)) & 0x0F0F0F0Fu;
    d = (d | (d << 2)) & 0x33333333u;
    const uint32_t lo_b = d & kNib;          // code bit 0: 1 -> j-1 / i-1
    const uint32_t hi_b = (d >> 1) & kNib;   // code bit 1: 1 -> vertical neighbour
    const uint32_t sx = PGG_Y(0, 0);
    const uint32_t sy = mux(hi_b, mux(lo_b, PGG_Y(0, 1), PGG_Y(0, -1)), mux(lo_b, PGG_Y(1, 0), PGG_Y(-1, 0)));
    const uint32_t active = (sx ^ sy) & u.msk;
    sx_out = sx;
    if (!active) return 0u;

    // group counts n(di, dj) of the groups centred within distance 2 of the sites
#define PGG_N(DI, DJ) (PGG_Y(DI, DJ) + PGG_Y(DI, (DJ) - 1) + PGG_Y(DI, (DJ) + 1) + PGG_Y((DI) - 1, DJ) + PGG_Y((DI) + 1, DJ))
    const uint32_t n00 = PGG_N(0, 0), n0e = PGG_N(0, 1), n0w = PGG_N(0, -1);
    const uint32_t n0ee = PGG_N(0, 2), n0ww = PGG_N(0, -2);
    const uint32_t ns0 = PGG_N(1, 0), nn0 = PGG_N(-1, 0);
    const uint32_t nse = PGG_N(1, 1), nsw = PGG_N(1, -1), nne = PGG_N(-1, 1), nnw = PGG_N(-1, -1);
    const uint32_t nss = PGG_N(2, 0), nnn = PGG_N(-2, 0);
#undef PGG_N
#undef PGG_Y
    // S = P + Q (nibble sums, P <= 15, Q <= 10)
    const uint32_t Px = n00 + n0w + n0e, Qx = nn0 + ns0;
    const uint32_t Pe = n0e + n00 + n0ee, Qe = nne + nse;   // y = (i, j+1)
    const uint32_t Pw = n0w + n0ww + n00, Qw = nnw + nsw;   // y = (i, j-1)
    const uint32_t Ps = ns0 + nsw + nse, Qs = n00 + nss;    // y = (i+1, j)
    const uint32_t Pn = nn0 + nnw + nne, Qn = nnn + n00;    // y = (i-1, j)
    const uint32_t lo_n = lo_b * 15u, hi_n = hi_b * 15u;
    const uint32_t Py = mux(hi_n, mux(lo_n, Pe, Pw), mux(lo_n, Ps, Pn));
    const uint32_t Qy = mux(hi_n, mux(lo_n, Qe, Qw), mux(lo_n, Qs, Qn));

    // bytes: even sites (m = 0, 2, 4, 6) and odd sites; A = s_x*26 + S_x <= 51
    const uint32_t Ae = (Px & kLowNib) + (Qx & kLowNib) + 26u * (sx & 0x01010101u);
    const uint32_t Ao = ((Px >> 4) & kLowNib) + ((Qx >> 4) & kLowNib) + 26u * ((sx >> 4) & 0x01010101u);
    const uint32_t Be = (Py & kLowNib) + (Qy & kLowNib);
    const uint32_t Bo = ((Py >> 4) & kLowNib) + ((Qy >> 4) & kLowNib);
    // halfword lanes: table index (s_x*26 + S_x)*26 + S_y <= 1351
    const uint32_t Ie01 = __byte_perm(Ae, 0u, 0x4140) * 26u + __byte_perm(Be, 0u, 0x4140);  // m = 0, 2
    const uint32_t Ie23 = __byte_perm(Ae, 0u, 0x4342) * 26u + __byte_perm(Be, 0u, 0x4342);  // m = 4, 6
    const uint32_t Io01 = __byte_perm(Ao, 0u, 0x4140) * 26u + __byte_perm(Bo, 0u, 0x4140);  // m = 1, 3
    const uint32_t Io23 = __byte_perm(Ao, 0u, 0x4342) * 26u + __byte_perm(Bo, 0u, 0x4342);  // m = 5, 7

    uint4 u0 = make_uint4(0, 0, 0, 0), u1 = make_uint4(0, 0, 0, 0);
    if (active & 0x0000FFFFu) u0 = draw_u4(u.seed, u.k, u.a, 2u * static_cast<uint32_t>(u.gw));
    if (active & 0xFFFF0000u) u1 = draw_u4(u.seed, u.k, u.a, 2u * static_cast<uint32_t>(u.gw) + 1u);

    uint32_t flips = 0;
#define PGG_SITE(M, IREG, HALF, UW)                                                 \
    if (active & (1u << (4 * (M)))) {                                               \
        const uint32_t idx = (IREG >> (16 * (HALF))) & 0xFFFFu;                     \
        if ((UW) < s_table[idx]) flips |= 1u << (4 * (M));                          \
    }
    PGG_SITE(0, Ie01, 0, u0.x)
    PGG_SITE(1, Io01, 0, u0.y)
    PGG_SITE(2, Ie01, 1, u0.z)
    PGG_SITE(3, Io01, 1, u0.w)
    PGG_SITE(4, Ie23, 0, u1.x)
    PGG_SITE(5, Io23, 0, u1.y)
    PGG_SITE(6, Ie23, 1, u1.z)
    PGG_SITE(7, Io23, 1, u1.w)
#undef PGG_SITE
    return flips;
}

// Periodic wrap of an index that may be a few periods outside [0, m).
__device__ __forceinline__ int wrap_small(int v, int m) {
    while (v < 0) v += m;
    while (v >= m) v -= m;
    return v;
}

// The part of the tile one fused step updates: sublattice rows r_first, r_first + 4, ...
// below row_hi, and local words [w_lo, w_hi) (sites outside [col_lo, col_hi) masked).
struct StepGeom {
    int row_hi, col_lo, col_hi, w_lo, w_hi, r_first, n_srows, n_words;
};

__device__ __forceinline__ StepGeom step_geom(const TiledParams &p, int ih, int iw, int j, int oi) {
    StepGeom g;
    const int e = 3 * (p.steps - 1 - j);
    const int row_lo = p.H - e;
    g.row_hi = p.H + ih + e;
    g.col_lo = 32 * p.hw - e;
    g.col_hi = 32 * p.hw + iw + e;
    g.w_lo = g.col_lo >> 5;
    g.w_hi = (g.col_hi + 31) >> 5;
    g.r_first = row_lo + ((oi + p.H - row_lo) & 3);
    g.n_srows = g.r_first < g.row_hi ? (g.row_hi - g.r_first + 3) >> 2 : 0;
    g.n_words = g.w_hi - g.w_lo;
    return g;
}

// Direction codes of step j for every unit of its region, into s_dir[srow * n_words + w]
// (16 bits per unit). One Philox call covers 64 sublattice sites = 8 words of a row, so a
// thread takes one row and one run of 8 words aligned to the global call boundary.
__device__ __forceinline__ void tile_dirs(const TiledParams &p, uint16_t *s_dir, int y0, int x0w,
                                          int ih, int iw, int j, int oi, int tid, int nthreads) {
    const StepGeom g = step_geom(p, ih, iw, j, oi);
    const uint64_t k = p.k0 + j;
    const int u_lo = x0w - p.hw + g.w_lo;          // unwrapped global word of w_lo
    const int c_lo = u_lo >> 3;                     // floor: first call-aligned run
    const int c_hi = (x0w - p.hw + g.w_hi - 1) >> 3;
    const int n_runs = c_hi - c_lo + 1;
    for (int t = tid; t < g.n_srows * n_runs; t += nthreads) {
        const int sr = t / n_runs;
        const int c = c_lo + (t - sr * n_runs);
        const int r = g.r_first + 4 * sr;
        const uint32_t a = static_cast<uint32_t>(wrap_small(y0 - p.H + r, p.L) >> 2);
        const int w0 = max(g.w_lo, 8 * c - (x0w - p.hw));
        const int w1 = min(g.w_hi, 8 * c + 8 - (x0w - p.hw));
        int cached = -1;
        uint4 call = make_uint4(0, 0, 0, 0);
        for (int w = w0; w < w1; ++w) {
            const int gw = wrap_small(x0w - p.hw + w, p.Lw);
            const int dg = gw >> 3;
            if (dg != cached) {
                call = philox4x32_10(static_cast<uint32_t>(dg), a, static_cast<uint32_t>(k),
                                     static_cast<uint32_t>(k >> 32) | kTagDir,
                                     static_cast<uint32_t>(p.seed), static_cast<uint32_t>(p.seed >> 32));
                cached = dg;
            }
            s_dir[sr * g.n_words + (w - g.w_lo)] =
                static_cast<uint16_t>(word_of(call, (gw >> 1) & 3) >> (16 * (gw & 1)));
        }
    }
}

// One sublattice step over the update region of the tile, for column offset OJ.
template <int LAYOUT, int WPT, int BLOCK, int OJ>
__device__ __forceinline__ void tile_step(const TiledParams &p, uint32_t *s_tile,
                                          const uint32_t *__restrict__ s_table,
                                          const uint16_t *__restrict__ s_dir, int y0, int x0w,
                                          int ih, int iw, int j, int oi) {
    const uint64_t k = p.k0 + j;
    const StepGeom g = step_geom(p, ih, iw, j, oi);
    const int n_wg = (g.n_words + WPT - 1) / WPT;
    const int n_tasks = g.n_srows * n_wg;
    const bool in_place = (p.steps == 1);

    for (int t = threadIdx.x; t < n_tasks; t += BLOCK) {
        const int sr = t / n_wg;
        const int wg = t - sr * n_wg;
        const int r = g.r_first + 4 * sr;
        const int wa = g.w_lo + wg * WPT;
        const int wb = min(wa + WPT, g.w_hi);
        const int grow = wrap_small(y0 - p.H + r, p.L);
        UnitCtx u;
        u.seed = p.seed;
        u.k = k;
        u.a = static_cast<uint32_t>(grow >> 2);

        uint32_t wl[7], wc[7], wr[7];
        const uint32_t *row0 = s_tile + (r - 3) * p.pitch;
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            wl[q] = row0[q * p.pitch + skew<WPT>(wa - 1)];
            wc[q] = row0[q * p.pitch + skew<WPT>(wa)];
        }
        int gw = wrap_small(x0w - p.hw + wa, p.Lw);
#pragma unroll
        for (int s = 0; s < WPT; ++s) {
            const int w = wa + s;
            if (w >= wb) break;
#pragma unroll
            for (int q = 0; q < 7; ++q) wr[q] = row0[q * p.pitch + skew<WPT>(w + 1)];
            u.gw = gw;
            u.d16 = s_dir[sr * g.n_words + (w - g.w_lo)];
            u.msk = kNib;
            if (w == g.w_lo || w == g.w_hi - 1) {
                // sites at local columns 32 w + OJ + 4 m inside [col_lo, col_hi)
                const int base = 32 * w + OJ;
                u.msk = nibble_range((g.col_lo - base + 3) >> 2, (g.col_hi - base + 3) >> 2);
            }
            uint32_t sx;
            const uint32_t flips = unit_flips<OJ>(wl, wc, wr, u, s_table, sx);
            if (flips) {
                const uint32_t nw = wc[3] ^ (flips << OJ);
                s_tile[r * p.pitch + skew<WPT>(w)] = nw;
                if (in_place) {
                    if (LAYOUT == kPacked) {
                        static_cast<uint32_t *>(p.dst)[static_cast<size_t>(grow) * p.Lw + gw] = nw;
                    } else {
                        uint8_t *rowp = static_cast<uint8_t *>(p.dst) + static_cast<size_t>(grow) * p.L + 32 * gw + OJ;
                        const uint32_t newbits = (sx ^ flips);
#pragma unroll
                        for (int m = 0; m < 8; ++m)
                            if (flips & (1u << (4 * m))) rowp[4 * m] = static_cast<uint8_t>((newbits >> (4 * m)) & 1u);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                wl[q] = wc[q];
                wc[q] = wr[q];
            }
            if (++gw == p.Lw) gw = 0;
        }
    }
}

template <int LAYOUT, int WPT, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_step_tiled(const TiledParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *s_table = smem;
    int *s_off = reinterpret_cast<int *>(smem + kTableEntries);
    uint16_t *s_dir = reinterpret_cast<uint16_t *>(smem + kTableEntries + kMaxSteps);
    uint32_t *s_tile = smem + kTableEntries + kMaxSteps + p.dir_words;
    __shared__ unsigned long long s_warp_count[BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = BLOCK / 32;

    for (int t = threadIdx.x; t < kTableEntries; t += BLOCK) s_table[t] = p.table[t];
    if (threadIdx.x < p.steps) s_off[threadIdx.x] = draw_offset(p.seed, p.k0 + threadIdx.x);

    const int n_tiles = p.tiles_x * p.tiles_y;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int ty = tile / p.tiles_x;
        const int tx = tile - ty * p.tiles_x;
        const int y0 = ty * p.tile_y, x0 = tx * p.tile_x;
        const int ih = min(p.tile_y, p.L - y0), iw = min(p.tile_x, p.L - x0);
        const int x0w = x0 >> 5;
        const int R = ih + 2 * p.H;
        const int Wr = (iw >> 5) + 2 * p.hw;
        __syncthreads();  // offsets ready; the previous tile is fully consumed
        // stage tile + halo as bit rows
        for (int r = warp; r < R; r += kWarps) {
            const int grow = wrap_small(y0 - p.H + r, p.L);
            for (int w = lane; w < Wr; w += 32) {
                const int gw = wrap_small(x0w - p.hw + w, p.Lw);
                uint32_t bits;
                if (LAYOUT == kPacked) {
                    bits = static_cast<const uint32_t *>(p.src)[static_cast<size_t>(grow) * p.Lw + gw];
                } else {
                    const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const uint8_t *>(p.src) +
                                                                       static_cast<size_t>(grow) * p.L + 32 * gw);
                    bits = pack32(src[0], src[1]);
                }
                s_tile[r * p.pitch + skew<WPT>(w)] = bits;
            }
        }
        tile_dirs(p, s_dir, y0, x0w, ih, iw, 0, s_off[0] >> 2, threadIdx.x, BLOCK);
        __syncthreads();
        for (int j = 0; j < p.steps; ++j) {
            const int o = s_off[j];
            const int oi = o >> 2;
            const uint16_t *dir_j = s_dir + (j & 1) * p.dir_slot;
            switch (o & 3) {
                case 0: tile_step<LAYOUT, WPT, BLOCK, 0>(p, s_tile, s_table, dir_j, y0, x0w, ih, iw, j, oi); break;
                case 1: tile_step<LAYOUT, WPT, BLOCK, 1>(p, s_tile, s_table, dir_j, y0, x0w, ih, iw, j, oi); break;
                case 2: tile_step<LAYOUT, WPT, BLOCK, 2>(p, s_tile, s_table, dir_j, y0, x0w, ih, iw, j, oi); break;
                default: tile_step<LAYOUT, WPT, BLOCK, 3>(p, s_tile, s_table, dir_j, y0, x0w, ih, iw, j, oi); break;
            }
            if (j + 1 < p.steps)
                tile_dirs(p, s_dir + ((j + 1) & 1) * p.dir_slot, y0, x0w, ih, iw, j + 1,
                          s_off[j + 1] >> 2, threadIdx.x, BLOCK);
            __syncthreads();
        }
        // write the interior back (fused launches) and count it
        unsigned long long cnt = 0;
        const int iwords = iw >> 5;
        for (int rr = warp; rr < ih; rr += kWarps) {
            for (int ww = lane; ww < iwords; ww += 32) {
                const uint32_t bits = s_tile[(p.H + rr) * p.pitch + skew<WPT>(p.hw + ww)];
                cnt += __popc(bits);
                if (p.steps > 1) {
                    const int grow = y0 + rr;
                    const int gw = x0w + ww;
                    if (LAYOUT == kPacked) {
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

int pitch_for(int wpt, int Wr) {
    int pitch = Wr + (Wr + wpt - 1) / wpt;
    if ((pitch & 1) == 0) ++pitch;
    return pitch;
}

// Largest region of one step: sublattice rows and words (for the direction buffer).
void dir_slot_dims(int steps, int tile_x, int tile_y, int *srows, int *words) {
    const int e = 3 * (steps - 1);
    *srows = (tile_y + 2 * e + 3) / 4 + 1;
    *words = (tile_x + 2 * e + 31) / 32 + 2;
}

size_t smem_bytes_for(int steps, int tile_x, int tile_y, int wpt, int *dir_slot, int *dir_words) {
    const int H = 3 * steps;
    const int hw = halo_words(steps);
    const int R = tile_y + 2 * H;
    const int Wr = tile_x / 32 + 2 * hw;
    int sr, ww;
    dir_slot_dims(steps, tile_x, tile_y, &sr, &ww);
    const int slot = sr * ww;                       // uint16 entries per step slot
    const int dwords = (2 * slot + 1) / 2 + 1;      // two slots, in uint32 words
    if (dir_slot) *dir_slot = slot;
    if (dir_words) *dir_words = (dwords + 3) & ~3;  // keep the tile 16-byte aligned
    return sizeof(uint32_t) * (static_cast<size_t>(kTableEntries) + kMaxSteps + ((dwords + 3) & ~3) +
                               static_cast<size_t>(R) * pitch_for(wpt, Wr));
}

template <int LAYOUT, int WPT>
cudaError_t launch_instance(const TiledParams &p, size_t smem, int grid, cudaStream_t s) {
    constexpr int kBlock = 256;
    auto kernel = k_step_tiled<LAYOUT, WPT, kBlock>;
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

// Words per thread task: small tiles need small tasks to keep all threads busy.
int pick_wpt(int tile_x, int tile_y) {
    const long tasks_wpt2 = static_cast<long>(tile_y / 4) * (tile_x / 64);
    return tasks_wpt2 >= 512 ? 2 : 1;
}

}  // namespace

size_t tiled_smem_bytes(int layout, int steps, int tile_x, int tile_y) {
    (void)layout;
    if (steps < 1 || steps > kMaxSteps || tile_x < 64 || tile_x % 64 || tile_y < 4 || tile_y % 4) return 0;
    const size_t b = smem_bytes_for(steps, tile_x, tile_y, pick_wpt(tile_x, tile_y), nullptr, nullptr);
    return b <= kMaxSmem ? b : 0;
}

cudaError_t launch_step_tiled(const TiledArgs &a, cudaStream_t s) {
    if (a.L < 64 || a.L % 64 || a.tile_x % 64 || a.tile_y % 4 || a.tile_x > a.L || a.tile_y > a.L)
        return cudaErrorInvalidValue;
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
    p.H = 3 * a.steps;
    p.hw = halo_words(a.steps);
    const int wpt = pick_wpt(a.tile_x, a.tile_y);
    p.pitch = pitch_for(wpt, a.tile_x / 32 + 2 * p.hw);
    p.table = a.table;
    p.count_out = a.count_out;
    const size_t smem = smem_bytes_for(a.steps, a.tile_x, a.tile_y, wpt, &p.dir_slot, &p.dir_words);
    if (smem > kMaxSmem) return cudaErrorInvalidValue;
    const int grid = p.tiles_x * p.tiles_y;
    if (a.layout == kPacked) {
        if (wpt == 2) return launch_instance<kPacked, 2>(p, smem, grid, s);
        return launch_instance<kPacked, 1>(p, smem, grid, s);
    }
    if (wpt == 2) return launch_instance<kU8, 2>(p, smem, grid, s);
    return launch_instance<kU8, 1>(p, smem, grid, s);
}

}  // namespace pgg
