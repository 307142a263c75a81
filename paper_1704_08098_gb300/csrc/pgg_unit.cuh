// pgg_unit.cuh -- the per-word update core shared by the lattice step kernels.
//
// Work unit: one 32-column word of one sublattice row. Its 8 sublattice sites sit at bits
// oj + 4m (m = 0..7), four bits apart, so after shifting the word's neighbourhood by oj
// every quantity of the 8 sites lives in one nibble of a 32-bit register:
//   Y(di, dj)    bit 4m = strategy of the site at (i + di, j_m + dj)
//   n(di, dj)    = Y(di,dj) + Y(di,dj-1) + Y(di,dj+1) + Y(di-1,dj) + Y(di+1,dj)
//                  the cooperator count of the group centred at (i+di, j_m+dj) (Fig. 1)
//   S(z)         = n(z) + n(z's 4 neighbours), kept as two partial nibble sums (<= 15, <= 10)
// S(x) and S(y) (y chosen by the direction draw) index the threshold table of Eq. (3); a
// site adopts s_y iff s_x != s_y and its adoption draw u is below the threshold.
#pragma once

#include <cstdint>

#include "pgg_device.cuh"

namespace pgg {

constexpr uint32_t kNib = 0x11111111u;
constexpr uint32_t kLowNib = 0x0F0F0F0Fu;

// The 32 columns starting D columns to the right (D < 0: left) of the word whose left,
// centre and right neighbours are l, c, r.
template <int D>
__device__ __forceinline__ uint32_t window(uint32_t l, uint32_t c, uint32_t r) {
    static_assert(D >= -6 && D <= 6, "window shift out of range");
    if constexpr (D == 0) return c;
    else if constexpr (D > 0) return __funnelshift_r(c, r, D);
    else return __funnelshift_l(l, c, -D);
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

// An opaque 1 in constant memory: x * c_one + y compiles to an integer multiply-add, issued on
// the FMA pipe, where x + y would go to the ALU pipe. The group-count sums below use it for two of
// their four additions, which balances the two pipes (the ALU pipe is otherwise the busier one:
// 72 M against 43 M warp instructions per MCS at L = 8192 before, 67 M against 54 M after).
static __constant__ uint32_t c_one = 1u;

// Threshold table entry at a byte offset (the unit cores build offsets, 4 x the index, in their
// packed lanes, which saves the scaling of each address).
__device__ __forceinline__ uint32_t table_at(const uint32_t *__restrict__ s_table, uint32_t off) {
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(s_table) + off);
}

struct UnitCtx {
    uint64_t k;
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
                                               const PhiloxKeys &rk,
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
#define PGG_N(DI, DJ) (PGG_Y(DI, DJ) + PGG_Y(DI, (DJ) - 1) + (PGG_Y(DI, (DJ) + 1) * c_one + (PGG_Y((DI) - 1, DJ) * c_one + PGG_Y((DI) + 1, DJ))))
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
    const uint32_t Be = ((Py & kLowNib) + (Qy & kLowNib)) * 4u;                 // 4 S_y <= 100
    const uint32_t Bo = (((Py >> 4) & kLowNib) + ((Qy >> 4) & kLowNib)) * 4u;
    // halfword lanes: byte offset of the table entry, 4 ((s_x*26 + S_x)*26 + S_y) <= 5404
    const uint32_t Ie01 = __byte_perm(Ae, 0u, 0x4140) * 104u + __byte_perm(Be, 0u, 0x4140);  // m = 0, 2
    const uint32_t Ie23 = __byte_perm(Ae, 0u, 0x4342) * 104u + __byte_perm(Be, 0u, 0x4342);  // m = 4, 6
    const uint32_t Io01 = __byte_perm(Ao, 0u, 0x4140) * 104u + __byte_perm(Bo, 0u, 0x4140);  // m = 1, 3
    const uint32_t Io23 = __byte_perm(Ao, 0u, 0x4342) * 104u + __byte_perm(Bo, 0u, 0x4342);  // m = 5, 7

    // adoption draws: call 2gw serves sites 0..3, call 2gw+1 sites 4..7. Both calls run
    // (interleaved) whenever the word has an active site: the lanes of a warp seldom need the
    // same halves, and one uniform path costs the warp two calls where per-lane choices cost
    // three (the divergent one-call and two-call paths one after the other)
    const uint32_t g0 = 2u * static_cast<uint32_t>(u.gw);
    const uint32_t kl = static_cast<uint32_t>(u.k), kh = static_cast<uint32_t>(u.k >> 32) | kTagU;
    uint4 u0 = make_uint4(g0, u.a, kl, kh), u1 = make_uint4(g0 + 1u, u.a, kl, kh);
    philox_rk2(u0, u1, rk);

    // every site looks its threshold up (all offsets lie inside the table) and the sites that
    // are not active are masked out once at the end: cheaper than a predicate per site
    uint32_t flips = 0;
#define PGG_SITE(M, IREG, HALF, UW)                                                 \
    {                                                                               \
        const uint32_t off = (IREG >> (16 * (HALF))) & 0xFFFFu;                     \
        flips |= ((UW) < table_at(s_table, off)) ? 1u << (4 * (M)) : 0u;            \
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
    return flips & active;
}

// The pairwise game (Section VI): every player plays a 2x2 game with each of its four
// nearest neighbours, so its payoff depends only on its strategy and the number of
// cooperating neighbours n (0..4), and an update reads the Manhattan ball of radius 2 (one
// line less than the group game; rows q = 1..5 of wl/wc/wr):
//   n(x)         = Y(0,1) + Y(0,-1) + Y(1,0) + Y(-1,0)
//   n(y), y = x + (0,1): Y(0,2) + Y(0,0) + Y(1,1) + Y(-1,1), and likewise for the others.
// The threshold table is indexed (s_x*5 + n_x)*5 + n_y (s_y = 1 - s_x where it is used).
template <int OJ>
__device__ __forceinline__ uint32_t unit_flips_pair(const uint32_t (&wl)[7], const uint32_t (&wc)[7],
                                                    const uint32_t (&wr)[7], const UnitCtx &u,
                                                    const PhiloxKeys &rk,
                                                    const uint32_t *__restrict__ s_table, uint32_t &sx_out) {
#define PGG_Y(DI, DJ) (window<(DJ) + OJ>(wl[(DI) + 3], wc[(DI) + 3], wr[(DI) + 3]) & kNib)
    uint32_t d = u.d16;
    d = (d | (d << 8)) & 0x00FF00FFu;
    d = (d | (d << 4)) & 0x0F0F0F0Fu;
    d = (d | (d << 2)) & 0x33333333u;
    const uint32_t lo_b = d & kNib;
    const uint32_t hi_b = (d >> 1) & kNib;
    const uint32_t sx = PGG_Y(0, 0);
    const uint32_t ye = PGG_Y(0, 1), yw = PGG_Y(0, -1), ys = PGG_Y(1, 0), yn = PGG_Y(-1, 0);
    const uint32_t sy = mux(hi_b, mux(lo_b, ye, yw), mux(lo_b, ys, yn));
    const uint32_t active = (sx ^ sy) & u.msk;
    sx_out = sx;
    if (!active) return 0u;

    const uint32_t nx = ye + yw + ys + yn;
    const uint32_t yse = PGG_Y(1, 1), ysw = PGG_Y(1, -1), yne = PGG_Y(-1, 1), ynw = PGG_Y(-1, -1);
    const uint32_t ne = PGG_Y(0, 2) + sx + yse + yne;   // y = (i, j+1)
    const uint32_t nw = PGG_Y(0, -2) + sx + ysw + ynw;  // y = (i, j-1)
    const uint32_t ns = PGG_Y(2, 0) + sx + yse + ysw;   // y = (i+1, j)
    const uint32_t nn = PGG_Y(-2, 0) + sx + yne + ynw;  // y = (i-1, j)
#undef PGG_Y
    const uint32_t lo_n = lo_b * 15u, hi_n = hi_b * 15u;
    const uint32_t ny = mux(hi_n, mux(lo_n, ne, nw), mux(lo_n, ns, nn));
    // bytes: even sites (m = 0, 2, 4, 6) and odd sites; byte offset 4 (25 s_x + 5 n_x + n_y) <= 196
    const uint32_t Ie = 100u * (sx & 0x01010101u) + 20u * (nx & kLowNib) + 4u * (ny & kLowNib);
    const uint32_t Io = 100u * ((sx >> 4) & 0x01010101u) + 20u * ((nx >> 4) & kLowNib) + 4u * ((ny >> 4) & kLowNib);

    // adoption draws: both calls whenever the word has an active site (as in unit_flips)
    const uint32_t g0 = 2u * static_cast<uint32_t>(u.gw);
    const uint32_t kl = static_cast<uint32_t>(u.k), kh = static_cast<uint32_t>(u.k >> 32) | kTagU;
    uint4 u0 = make_uint4(g0, u.a, kl, kh), u1 = make_uint4(g0 + 1u, u.a, kl, kh);
    philox_rk2(u0, u1, rk);

    uint32_t flips = 0;
#define PGG_SITE(M, IREG, BYTE, UW)                                                 \
    {                                                                               \
        const uint32_t off = (IREG >> (8 * (BYTE))) & 0xFFu;                        \
        flips |= ((UW) < table_at(s_table, off)) ? 1u << (4 * (M)) : 0u;            \
    }
    PGG_SITE(0, Ie, 0, u0.x)
    PGG_SITE(1, Io, 0, u0.y)
    PGG_SITE(2, Ie, 1, u0.z)
    PGG_SITE(3, Io, 1, u0.w)
    PGG_SITE(4, Ie, 2, u1.x)
    PGG_SITE(5, Io, 2, u1.y)
    PGG_SITE(6, Ie, 3, u1.z)
    PGG_SITE(7, Io, 3, u1.w)
#undef PGG_SITE
    return flips & active;
}

template <int OJ, int GAME>
__device__ __forceinline__ uint32_t game_flips(const uint32_t (&wl)[7], const uint32_t (&wc)[7],
                                               const uint32_t (&wr)[7], const UnitCtx &u,
                                               const PhiloxKeys &rk,
                                               const uint32_t *__restrict__ s_table, uint32_t &sx_out) {
    if constexpr (GAME == kPairGame) return unit_flips_pair<OJ>(wl, wc, wr, u, rk, s_table, sx_out);
    else return unit_flips<OJ>(wl, wc, wr, u, rk, s_table, sx_out);
}

// Rows q (0..6, row offsets -3..+3) a game's update reads.
template <int GAME>
__host__ __device__ constexpr bool reads_row(int q) {
    return q >= 3 - kReadRadius<GAME> && q <= 3 + kReadRadius<GAME>;
}

// Periodic wrap of an index that may be a few periods outside [0, m).
__device__ __forceinline__ int wrap_small(int v, int m) {
    while (v < 0) v += m;
    while (v >= m) v -= m;
    return v;
}

}  // namespace pgg
