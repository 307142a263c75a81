// pgg_kernels_resident.cu -- a whole bit-packed lattice resident in shared memory across
// many MCS: one cooperative launch, each CTA owning a band of rows.
//
// CTA b keeps rows [r0, r0 + nb) of the lattice plus H halo rows above and below in shared
// memory for the whole call. A sublattice step writes only rows i = oi (mod 4), at least 4
// apart, and an update reads the Manhattan ball of radius R around its site (R = 3 for the
// group game, Section IV, Fig. 3; R = 2 for the pairwise game of Section VI), so within a
// step no CTA needs data a neighbour writes in that step.
//
// Halo exchange every s steps (s = 1, 2 or 4; H = R s). The CTA updates, at step j of a
// block of s steps, the sublattice rows of its band and of the R (s - 1 - j) halo rows next to
// it on each side: the halo rows are its neighbours' band rows, updated redundantly with the
// same counter-based draws, so after the block the band is exact and only the neighbours'
// H edge rows must be fetched again. After each block the CTA publishes its top and bottom H
// band rows to a double-buffered mailbox in global memory and bumps its block counter; before
// the rows that read the halo in the first step of the next block it waits for both
// neighbours' counters and their rows in its halo. All CTAs are co-resident (cooperative
// launch). Every wait is bounded: after `spin_limit` polls the CTA sets the status word and
// stops; its neighbours then time out in turn.
//
// The exchange runs beside the computation: one extra warp per CTA polls the neighbours'
// counters, fetches their edge rows into the halo with TMA bulk copies (cp.async.bulk,
// completion on an mbarrier) and bulk-stores the band's own edge rows and releases its counter,
// while the 16 compute warps update the rows that do not read the halo; the compute warps wait on
// the mbarrier only before the rows that do. With s > 1 the last step of a block (band rows
// only, no halo wait) updates the top and bottom H rows first and hands them over through a named
// barrier, so they go out while the rows between them are updated; the exchange warp's copy has
// read them before the step ends, after which they change again. With s = 1 they go out after
// the step: the next step touches them only after its own halo wait, which follows the copy.
//
// Where shared memory allows (the group game), the CTA also keeps its rows as a column-class copy,
// 32 sites of one column class j mod 4 per word, and scans that for the active sites of a step;
// adoptions flip both copies and the exchange carries both (see the class-copy helpers below). The
// lattice's class copy stays in global memory between launches (cls_g): a launch stages it while it
// holds the lattice and builds it from the rows otherwise, and writes the band's part back.
//
// Work within a step: most sites of a sublattice step cannot change, because an update with
// s_x = s_y is a no-op (Eq. (3) only matters when the strategies differ) and needs no adoption
// draw (the stream is counter based). Each warp therefore scans words of its sublattice rows
// (32 sites per class-word of the step's column class; without the class copy 8 sites per
// 32-column word, the direction draws of 8 words from one Philox call), finds the active sites
// (s_x != s_y for the drawn neighbour y), and appends them to a ring in shared memory (without
// the class copy active words first, then their sites); whenever 32 sites are waiting, the warp updates
// them, one per lane: the group counts S_x and S_y from the 7 x 7 neighbourhood of x (population
// counts of masked bits), the threshold of Eq. (3) from the host-built table, the adoption draw,
// and an atomic XOR of the site's bit when it adopts. So the costly part runs at full warp width
// on active sites only. When many sites are active (a random start, the pairwise game), a dense
// pass does better: every word, all 8 sites at once, by the shared per-word core of
// pgg_unit.cuh. Each step takes one pass or the other, chosen from the number of adoptions in
// the CTA's previous step; both give the same result. Updates of one step touch disjoint sites
// and read only bits no other update of the step changes, so they run in place in any order.
//
// The count after each MCS is the sum of the bands' population counts, gathered in count slots
// by the last band to report. The band is staged with 4-byte cp.async copies and written back once
// per launch; a uint8 lattice is packed as its band is staged (two 16-byte loads per word) and
// unpacked as it is written back, so it needs no conversion launches.
#include <cuda_runtime.h>

#include "pgg_device.cuh"
#include "pgg_internal.h"
#include "pgg_unit.cuh"

namespace pgg {
namespace {

constexpr int kComputeThreads = 512;                  // warps that update the band
constexpr int kComputeWarps = kComputeThreads / 32;
constexpr int kResThreads = kComputeThreads + 32;      // plus one warp that exchanges halos
constexpr int kMaxStepsPerExchange = 4;
constexpr int kMaxHalo = 3 * kMaxStepsPerExchange;    // halo rows per side at most
constexpr int kMaxLocalRows = 128;                     // band + halo rows (7 bits of a word entry)
constexpr int kMaxRowWords = 512;                      // words per row (9 bits of a word entry)

struct ResidentParams {
    uint32_t *lat;            // bit-packed global lattice (read at the start, written at the end)
    uint8_t *lat8;            // or, when not null, a uint8 lattice (lat unused)
    int L, Lw, n_bands;
    int s, H;                 // sublattice steps per halo exchange, halo rows per side (R s)
    uint64_t seed, k0;
    int n_mcs;
    const uint32_t *table;
    uint32_t *mailbox;        // [band][parity][top/bottom][H rows][Lw]
    unsigned int *ctr;        // [band] ctr_base + blocks published in this launch
    unsigned int ctr_base;    // above every value an earlier launch left in ctr
    unsigned long long *counts;  // [n_mcs], written by the launch
    unsigned long long *count_acc;  // [kResidentCountSlots] band-count sums, zero between launches
    unsigned int *count_tick;       // [kResidentCountSlots] bands that added to the sum, zero between launches
    int *status;              // | 1 a wait timed out, | 2 misaligned buffers, | 4 an index check failed (checked build),
                              // | 8 a CTA stopped with a halo load possibly still in flight
    unsigned int spin_limit;
    unsigned int *hint;       // [band] adoptions of the last step of the previous launch (nullable)
    unsigned int dense_per_mille;  // dense pass above this share (per mille) of a step's sites flipped
    uint32_t *cls_g;          // the lattice's column-class copy in global memory (CLS, nullable): written
                              // back with the band, and
    int cls_load;             // staged from there when it holds this lattice (else built from the rows)
    PhiloxKeys rk;
};

// Four bytes, each 0 or 1, to four bits (byte i to bit i): the product puts byte i's bit at
// bit 24 + i, and no two partial products share a bit position, so nothing carries.
__device__ __forceinline__ uint32_t pack_bytes4(uint32_t x) { return (x * 0x01020408u) >> 24; }

// 32 bytes of a uint8 row (0 or 1 each) to the bit-packed word (byte b to bit b).
__device__ __forceinline__ uint32_t pack_bytes32(const uint4 &a, const uint4 &b) {
    return pack_bytes4(a.x) | pack_bytes4(a.y) << 4 | pack_bytes4(a.z) << 8 | pack_bytes4(a.w) << 12 |
           pack_bytes4(b.x) << 16 | pack_bytes4(b.y) << 20 | pack_bytes4(b.z) << 24 | pack_bytes4(b.w) << 28;
}

// Four bits to four bytes of 0 or 1 (bit i to byte i): the product puts bit i at bit 8 i, and no
// two partial products share a bit position.
__device__ __forceinline__ uint32_t unpack_bits4(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }

__device__ __forceinline__ uint4 unpack_bits16(uint32_t h) {
    return make_uint4(unpack_bits4(h & 15u), unpack_bits4((h >> 4) & 15u), unpack_bits4((h >> 8) & 15u),
                      unpack_bits4((h >> 12) & 15u));
}

__device__ __forceinline__ int band_start(int b, int L, int n) { return static_cast<int>((static_cast<long long>(b) * L) / n); }

// Word w of a band row lives at (w ^ ((w >> 5) & 7)): lanes that read words 1, 2, 4 or 8 apart
// (words u c, c = 0..31) then hit 32 different banks.
__device__ __forceinline__ int swz(int w) { return w ^ ((w >> 5) & 7); }

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Named barrier 2: in the last step of a block the compute warps hand the band's edge rows over
// (arrive, without waiting) once they are updated, and the exchange warp waits for all of them.
__device__ __forceinline__ void edges_arrive() { asm volatile("bar.arrive 2, %0;" ::"n"(kResThreads) : "memory"); }
__device__ __forceinline__ void edges_wait() { asm volatile("bar.sync 2, %0;" ::"n"(kResThreads) : "memory"); }

__device__ __forceinline__ unsigned int load_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// --- the 7 x 7 neighbourhood of a site, one byte per row ------------------------------------
// Byte r holds row offset r - 3 and bit t of it column offset t - 3 (t = 7, column offset +4, is
// carried along and never used); the site itself is bit 27. Relative to a centre at bit 27, the
// group count sum of Section III, S = sum of the 5 group counts of the groups the centre belongs
// to (Fig. 1), weighs the centre 5 times, its 4 nearest neighbours and 4 diagonal neighbours
// twice, and the 4 sites two steps away along the axes once (a neighbour w of z lies in z's own
// group and in w's; a diagonal site in the groups of the two neighbours it shares with z; an axis
// site at distance 2 in the group of the neighbour between them).
constexpr uint32_t kOnesLo = (1u << 11) | (1u << 25) | (1u << 29);    // (-2, 0), (0, -2), (0, +2)
constexpr uint32_t kOnesHi = 1u << (43 - 32);                         // (+2, 0)
constexpr uint32_t kTwosLo = (1u << 18) | (1u << 19) | (1u << 20) | (1u << 26) | (1u << 28);
constexpr uint32_t kTwosHi = (1u << (34 - 32)) | (1u << (35 - 32)) | (1u << (36 - 32));  // row +1
// the 4 nearest neighbours alone (the pairwise game's cooperating neighbours, Section VI)
constexpr uint32_t kNearLo = (1u << 19) | (1u << 26) | (1u << 28);
constexpr uint32_t kNearHi = 1u << (35 - 32);

// --- the column-class copy ----------------------------------------------------------------
// Beside the bit-packed rows the kernel can keep a second copy of its rows in which a word holds
// 32 sites of one column class: class-word (c, q) of a row holds columns 128 q + 4 t + c at bit t
// (t = 0..31), at cls[lr * Lw + c * Lq + q] (Lq = Lw / 4). A sublattice step updates sites of one
// column class only, so a class-word carries 32 of them, their east and west neighbours sit in the
// neighbouring classes of the row (class 3 -> 0 one bit along) and the sites above and below in the
// same class-word of the rows around.

__device__ __forceinline__ uint32_t unshuffle_step(uint32_t x, int sft, uint32_t m) {
    const uint32_t t = ((x >> sft) ^ x) & m;
    return x ^ t ^ (t << sft);
}

// Bit 2 t of x to bit t, bit 2 t + 1 to bit 16 + t (t = 0..15): an outer unshuffle by delta swaps.
__device__ __forceinline__ uint32_t unzip32(uint32_t x) {
    x = unshuffle_step(x, 1, 0x22222222u);
    x = unshuffle_step(x, 2, 0x0C0C0C0Cu);
    x = unshuffle_step(x, 4, 0x00F000F0u);
    return unshuffle_step(x, 8, 0x0000FF00u);
}

// The class bytes of a bit-packed word (column b at bit b): byte 0 = columns 0, 4, .., 28 (class
// 0), byte 1 = class 2, byte 2 = class 1, byte 3 = class 3 (an outer unshuffle, then one within
// each half).
__device__ __forceinline__ uint32_t class_bytes(uint32_t w) {
    w = unzip32(w);
    w = unshuffle_step(w, 1, 0x22222222u);
    w = unshuffle_step(w, 2, 0x0C0C0C0Cu);
    return unshuffle_step(w, 4, 0x00F000F0u);
}

// Bits 4 m of f (m = 0..7) to bits m.
__device__ __forceinline__ uint32_t nibble_bits8(uint32_t f) {
    f = (f | (f >> 3)) & 0x03030303u;
    f = (f | (f >> 6)) & 0x000F000Fu;
    return (f | (f >> 12)) & 0xFFu;
}

// The class copy of n_rows rows: thread tid of nthr takes groups of 4 bit-packed words (one
// class-word of each class).
__device__ __forceinline__ void build_class_rows(const uint32_t *rows, uint32_t *cls, int n_rows, int Lw, int tid, int nthr,
                                                 int *status) {
    const int Lq = Lw >> 2;
    const long long n_words = static_cast<long long>(n_rows) * Lw;
    for (int g = tid; g < n_rows * Lq; g += nthr) {
        const int lr = g / Lq, qq = g - lr * Lq;
        const long long base = static_cast<long long>(lr) * Lw;
        uint32_t u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            u[k] = index_ok(base + swz(4 * qq + k), n_words, status) ? class_bytes(rows[base + swz(4 * qq + k)]) : 0u;
        if (!index_ok(base + 3 * Lq + qq, n_words, status)) continue;
        uint32_t *cr = cls + base + qq;
        cr[0] = __byte_perm(__byte_perm(u[0], u[1], 0x0040u), __byte_perm(u[2], u[3], 0x0040u), 0x5410u);
        cr[2 * Lq] = __byte_perm(__byte_perm(u[0], u[1], 0x0051u), __byte_perm(u[2], u[3], 0x0051u), 0x5410u);
        cr[Lq] = __byte_perm(__byte_perm(u[0], u[1], 0x0062u), __byte_perm(u[2], u[3], 0x0062u), 0x5410u);
        cr[3 * Lq] = __byte_perm(__byte_perm(u[0], u[1], 0x0073u), __byte_perm(u[2], u[3], 0x0073u), 0x5410u);
    }
}

struct Ctx {
    uint32_t *rows;                       // band + halo rows (local row lr = global row r0 - H + lr)
    uint32_t *cls;                        // their column-class copy (class-copy kernel only)
    int Lq;                               // class-words per class and row (Lw / 4)
    int cprq;                             // 32-class-word chunks per row
    uint32_t cmagicq;                     // ceil(2^16 / cprq)
    const uint32_t *__restrict__ table;
    int L, Lw, r0, H;
    uint32_t kl, kh_dir, kh_u;            // step index words with the direction / adoption tags
    const PhiloxKeys *rk;
    int cpr;                              // 64-word chunks per row
    uint32_t cmagic;                      // ceil(2^16 / cpr): floor(k / cpr) = (k cmagic) >> 16 for small k
    long long n_words;                    // words of band + halo rows (checked build)
    int *status;
    uint64_t k;                           // sublattice step index
    int oj;                               // column offset of the step's sublattice (0..3)
};

// The adoption decision of one active site: entry = local row << 18 | column << 2 | direction
// code. Returns the bit to flip (0: no adoption) and sets `word` to the index of its word in
// the band rows.
template <int GAME>
__device__ __forceinline__ uint32_t site_flip(const Ctx &cx, uint32_t e, int &word) {
    const int d = static_cast<int>(e & 3u);
    const int j = static_cast<int>((e >> 2) & 0xFFFFu);
    const int lr = static_cast<int>(e >> 18);
    int i = cx.r0 - cx.H + lr;
    if (i < 0) i += cx.L;
    else if (i >= cx.L) i -= cx.L;
    // adoption draw of sublattice site (a, b) = (i >> 2, j >> 2): word b & 3 of the call at b >> 2
    uint4 u4 = make_uint4(static_cast<uint32_t>(j >> 4), static_cast<uint32_t>(i >> 2), cx.kl, cx.kh_u);
#pragma unroll
    for (int r = 0; r < 10; ++r) philox_round(u4, cx.rk->k0[r], cx.rk->k1[r]);
    // columns j - 3 .. j + 4 of rows lr - 3 .. lr + 3, from the two words holding them
    const int c0 = j >= 3 ? j - 3 : j - 3 + cx.L;
    const int wa = c0 >> 5, wb = wa + 1 == cx.Lw ? 0 : wa + 1, sh = c0 & 31;
    constexpr int q0 = 3 - kReadRadius<GAME>;  // the rows the game reads: q0 .. 6 - q0
    const uint32_t *pa = cx.rows + swz(wa) + (lr - 3 + q0) * cx.Lw;
    const uint32_t *pb = cx.rows + swz(wb) + (lr - 3 + q0) * cx.Lw;
    uint32_t v[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const long long ra = static_cast<long long>(lr - 3 + q) * cx.Lw;
        v[q] = (q >= q0 && q <= 6 - q0 && index_ok(ra + swz(wa), cx.n_words, cx.status) &&
                index_ok(ra + swz(wb), cx.n_words, cx.status))
                   ? __funnelshift_r(pa[(q - q0) * cx.Lw], pb[(q - q0) * cx.Lw], sh)
                   : 0u;
    }
    // the rows' low bytes side by side: lo = rows 0..3, hi = rows 4..6 (its top byte is not used)
    const uint32_t lo = __byte_perm(__byte_perm(v[0], v[1], 0x0040u), __byte_perm(v[2], v[3], 0x0040u), 0x5410u);
    const uint32_t hi = __byte_perm(__byte_perm(v[4], v[5], 0x0040u), v[6], 0x0410u);
    const uint32_t sx = (lo >> 27) & 1u;
    // the same bits centred on y: shifted right for y to the right (+1) or below (+8), left otherwise
    const uint32_t rs = d == 0 ? 1u : (d == 2 ? 8u : 0u);
    const uint32_t ls = d == 1 ? 1u : (d == 3 ? 8u : 0u);
    uint32_t ylo = __funnelshift_r(lo, hi, rs), yhi = hi >> rs;
    yhi = __funnelshift_l(ylo, yhi, ls);
    ylo <<= ls;
    uint32_t idx;
    if constexpr (GAME == kPairGame) {
        const uint32_t nx = __popc(lo & kNearLo) + __popc(hi & kNearHi), ny = __popc(ylo & kNearLo) + __popc(yhi & kNearHi);
        idx = (sx * 5u + nx) * 5u + ny;
    } else {
        const uint32_t Sx = __popc(lo & kOnesLo) + __popc(hi & kOnesHi) +
                            2u * (__popc(lo & kTwosLo) + __popc(hi & kTwosHi)) + 5u * sx;
        const uint32_t Sy = __popc(ylo & kOnesLo) + __popc(yhi & kOnesHi) +
                            2u * (__popc(ylo & kTwosLo) + __popc(yhi & kTwosHi)) + 5u * (1u - sx);
        idx = (sx * 26u + Sx) * 26u + Sy;
    }
    const uint32_t t = index_ok(idx, kTableEntries, cx.status) ? cx.table[idx] : 0u;
    const int bw = (j >> 2) & 3;
    const uint32_t u = bw == 0 ? u4.x : bw == 1 ? u4.y : bw == 2 ? u4.z : u4.w;
    word = lr * cx.Lw + swz(j >> 5);
    return u < t && index_ok(word, cx.n_words, cx.status) ? 1u << (j & 31) : 0u;
}

// The rings of one warp: active words found by the scan, and the active sites they hold.
constexpr int kWordRingCap = 64;     // uint2 entries: (activity nibbles, lr << 25 | w << 16 | d16)
constexpr uint32_t kWordRingMask = kWordRingCap - 1;
constexpr int kSiteRingCap = 512;    // uint32 entries: lr << 18 | j << 2 | direction (< 32 + 256 held)
constexpr uint32_t kSiteRingMask = kSiteRingCap - 1;

struct Rings {
    uint2 *words;
    uint32_t *sites;
    uint32_t wh, wt, sh, st;  // heads and tails (warp-uniform)
    uint32_t flips;           // adoptions this thread made in the current step
};

// Warp-uniform: update the next n (<= 32) active sites, one per lane. A round is latency bound
// (the Philox draw and the neighbourhood gather of one site), so rounds of one site per lane end
// sooner than rounds of two, and a step's last, partial round is the shortest possible; sites of
// one step never read each other's bits, so the order does not matter.
// CLS: the kernel keeps the column-class copy, which an adoption flips too.
template <int GAME, bool CLS>
__device__ __forceinline__ void drain_sites(const Ctx &cx, Rings &q, uint32_t n, int lane) {
    __syncwarp();
    const uint32_t l = static_cast<uint32_t>(lane);
    if (l < n) {
        int a0;
        const uint32_t e0 = q.sites[(q.sh + l) & kSiteRingMask];
        const uint32_t f0 = site_flip<GAME>(cx, e0, a0);
        if (f0) {
            atomicXor(&cx.rows[a0], f0);
            if constexpr (CLS) {
                const uint32_t j = (e0 >> 2) & 0xFFFFu;
                const long long ci = static_cast<long long>(e0 >> 18) * cx.Lw + (j & 3u) * cx.Lq + (j >> 7);
                if (index_ok(ci, cx.n_words, cx.status)) atomicXor(&cx.cls[ci], 1u << ((j >> 2) & 31u));
            }
        }
        q.flips += f0 != 0u;
    }
    q.sh += n;
}

// Warp-uniform: turn the next n (<= 32) active words into site entries, one word per lane (the
// ring positions from a prefix sum of the lanes' site counts, <= 8, by its bits), then update
// sites while 32 or more are waiting. The site ring holds < 32 entries before and at most
// 31 + 256 after.
template <int GAME>
__device__ __forceinline__ void expand_words(const Ctx &cx, Rings &q, uint32_t n, int lane) {
    __syncwarp();
    uint32_t act = 0, y = 0;
    if (static_cast<uint32_t>(lane) < n) {
        const uint2 e = q.words[(q.wh + lane) & kWordRingMask];
        act = e.x;
        y = e.y;
    }
    q.wh += n;
    const uint32_t c = __popc(act), lt = (1u << lane) - 1u;
    const uint32_t b0 = __ballot_sync(0xffffffffu, c & 1u), b1 = __ballot_sync(0xffffffffu, c & 2u);
    const uint32_t b2 = __ballot_sync(0xffffffffu, c & 4u), b3 = __ballot_sync(0xffffffffu, c & 8u);
    uint32_t pos = q.st + __popc(b0 & lt) + 2u * __popc(b1 & lt) + 4u * __popc(b2 & lt) + 8u * __popc(b3 & lt);
    q.st += __popc(b0) + 2u * __popc(b1) + 4u * __popc(b2) + 8u * __popc(b3);
    const uint32_t d16 = y & 0xFFFFu;
    const uint32_t ebase = (y >> 25) << 18 | (32u * ((y >> 16) & 0x1FFu) + static_cast<uint32_t>(cx.oj)) << 2;
    while (act) {
        const int m = (__ffs(act) - 1) >> 2;
        q.sites[pos & kSiteRingMask] = ebase + (static_cast<uint32_t>(4 * m) << 2) + ((d16 >> (2 * m)) & 3u);
        ++pos;
        act &= act - 1u;
    }
    while (q.st - q.sh >= 32u) drain_sites<GAME, false>(cx, q, 32u, lane);
}

// Activity of the 8 sites of one word (nibble bits): s_x != s_y for the drawn neighbour y; oj: the
// sublattice's column offset. l, c, r:
// the word and its left and right neighbours in the site's row; uc, ur / dc, dr: the word and
// its right neighbour in the rows above / below; d16: the sites' direction codes.
__device__ __forceinline__ uint32_t word_activity(int oj, uint32_t l, uint32_t c, uint32_t r, uint32_t uc, uint32_t ur,
                                                  uint32_t dc, uint32_t dr, uint32_t d16) {
    uint32_t dd = d16;
    dd = (dd | (dd << 8)) & 0x00FF00FFu;
    dd = (dd | (dd << 4)) & 0x0F0F0F0Fu;
    dd = (dd | (dd << 2)) & 0x33333333u;
    const uint32_t lo_b = dd & kNib, hi_b = (dd >> 1) & kNib;
    // columns oj + 4m + D of the three rows (a shift of 0 returns the word itself)
    const uint32_t sx = __funnelshift_r(c, r, oj) & kNib;
    const uint32_t ye = __funnelshift_r(c, r, oj + 1) & kNib;
    const uint32_t yw = (oj ? __funnelshift_r(c, r, oj - 1) : __funnelshift_l(l, c, 1)) & kNib;
    const uint32_t ys = __funnelshift_r(dc, dr, oj) & kNib;
    const uint32_t yn = __funnelshift_r(uc, ur, oj) & kNib;
    return sx ^ mux(hi_b, mux(lo_b, ye, yw), mux(lo_b, ys, yn));
}

// Warp-uniform: append the lanes' active words to the word ring; expand 32 when they are there.
template <int GAME>
__device__ __forceinline__ void push_word(const Ctx &cx, Rings &q, uint32_t act, int lr, int w, uint32_t d16,
                                          int lane) {
    const uint32_t bal = __ballot_sync(0xffffffffu, act != 0u);
    if (act)
        q.words[(q.wt + __popc(bal & ((1u << lane) - 1u))) & kWordRingMask] =
            make_uint2(act, static_cast<uint32_t>(lr) << 25 | static_cast<uint32_t>(w) << 16 | d16);
    q.wt += __popc(bal);
    if (q.wt - q.wh >= 32u) expand_words<GAME>(cx, q, 32u, lane);
}

// Sublattice rows (local lr = first + 4 k, k < n) of a step.
struct Range {
    int first, n;
};

// The sublattice rows of the current step among local rows [lo, hi) (m4: lr = m4 (mod 4)).
__device__ __forceinline__ Range srows_in(int m4, int lo, int hi) {
    Range r{0, 0};
    if (hi <= lo) return r;
    r.first = lo + ((m4 - lo) & 3);
    r.n = r.first < hi ? (hi - r.first + 3) >> 2 : 0;
    return r;
}

// One 64-word chunk of a sublattice row as a lane sees it: its two words, their neighbours and
// their direction bits.
struct Chunk {
    int lr, wa;
    bool valid;
    uint32_t d32, cl, ca, cb, cq, ua, ub, uq, da, db, dq;
};

// The direction draws of a warp's next 4 chunks: lane l computes call l mod 8 of chunk o + l / 8
// (row lr2, column chunk c2; `have` false: past the warp's last chunk).
__device__ __forceinline__ void direction_calls(const Ctx &cx, uint4 &dcall, bool have, int lr2, int c2, int lane) {
    uint32_t g = 0, a = 0;
    if (have) {
        int i2 = cx.r0 - cx.H + lr2;
        if (i2 < 0) i2 += cx.L;
        else if (i2 >= cx.L) i2 -= cx.L;
        g = static_cast<uint32_t>(8 * c2 + (lane & 7));
        a = static_cast<uint32_t>(i2 >> 2);
    }
    dcall = make_uint4(g, a, cx.kl, cx.kh_dir);
#pragma unroll
    for (int rr = 0; rr < 10; ++rr) philox_round(dcall, cx.rk->k0[rr], cx.rk->k1[rr]);
}

// Load chunk (row ch.lr, column chunk c) of the warp's chunk ordinal o: words w0 = 64 c + 2 lane
// and w0 + 1. Their 32 direction bits are word lane mod 4 of call (chunk o, lane / 4), which
// lane 8 (o mod 4) + lane / 4 holds.
__device__ __forceinline__ void load_chunk(const Ctx &cx, const uint4 &dcall, int o, int c, int lane, Chunk &ch) {
    const int src = 8 * (o & 3) + (lane >> 2);
    const uint32_t dx = __shfl_sync(0xffffffffu, dcall.x, src), dy = __shfl_sync(0xffffffffu, dcall.y, src);
    const uint32_t dz = __shfl_sync(0xffffffffu, dcall.z, src), dw = __shfl_sync(0xffffffffu, dcall.w, src);
    const int comp = lane & 3;
    ch.d32 = comp == 0 ? dx : comp == 1 ? dy : comp == 2 ? dz : dw;
    const int w0 = 64 * c + 2 * lane;
    ch.valid = w0 < cx.Lw;  // Lw is even, so w0 + 1 is valid with w0
    ch.wa = ch.valid ? w0 : 0;
    const int wa = ch.wa;
    const int wp = wa == 0 ? cx.Lw - 1 : wa - 1, wb = wa + 1, wq = wa + 2 == cx.Lw ? 0 : wa + 2;
    const long long rb = static_cast<long long>(ch.lr - 1) * cx.Lw;
    const uint32_t *row = cx.rows + (ch.lr - 1) * cx.Lw;
#define PGG_LD(RR, WW) \
    (index_ok(rb + (RR) * cx.Lw + swz(WW), cx.n_words, cx.status) ? row[(RR) * cx.Lw + swz(WW)] : 0u)
    ch.cl = PGG_LD(1, wp);
    ch.ca = PGG_LD(1, wa);
    ch.cb = PGG_LD(1, wb);
    ch.cq = PGG_LD(1, wq);
    ch.ua = PGG_LD(0, wa);
    ch.ub = PGG_LD(0, wb);
    ch.uq = cx.oj > 0 ? PGG_LD(0, wq) : 0u;
    ch.da = PGG_LD(2, wa);
    ch.db = PGG_LD(2, wb);
    ch.dq = cx.oj > 0 ? PGG_LD(2, wq) : 0u;
#undef PGG_LD
}

// Scan the rows of up to three ranges in chunks of 64 words, two consecutive words per lane;
// chunk K of the ranges' concatenation goes to warp K mod 16, so the warps get equal shares.
// Before its first chunk in range wait_at or later the warp waits for the halo (`wait` returns
// false if it never lands), and at the end if it had no such chunk. Active words go to the
// warp's word ring, and 32 of them at a time to the site ring. The direction draws of a warp's
// next 4 chunks come from one Philox call per lane (chunk o + lane / 8, call lane mod 8 of the
// chunk's 8) and reach the lanes that use them by shuffles. Warp-uniform.
template <int GAME, class Wait>
__device__ __forceinline__ bool scan_step(const Ctx &cx, const Range (&rg)[3], int wait_at, Wait wait, Rings &q,
                                          int warp, int lane) {
    const int cpr = cx.cpr;
    const int n0 = rg[0].n * cpr, n1 = rg[1].n * cpr, total = n0 + n1 + rg[2].n * cpr;
    bool waited = wait_at < 0;
    uint4 dcall = make_uint4(0, 0, 0, 0);
    // row of chunk K and its column chunk
    auto locate = [&](int K, int &lr, int &c) -> int {
        int r = 0, kk = K;
        if (kk >= n0) {
            kk -= n0;
            r = 1;
            if (kk >= n1) {
                kk -= n1;
                r = 2;
            }
        }
        const int qr = static_cast<int>((static_cast<uint32_t>(kk) * cx.cmagic) >> 16);
        c = kk - qr * cpr;
        lr = (r == 0 ? rg[0].first : r == 1 ? rg[1].first : rg[2].first) + 4 * qr;  // no indexed array
        return r;
    };
    // two chunks per iteration (this warp's chunks o and o + 1): their loads and activity chains are
    // independent, which gives the scheduler two chains per warp to interleave
    int o = 0;
    for (int K = warp; K < total; K += 2 * kComputeWarps, o += 2) {
        const bool two = K + kComputeWarps < total;
        Chunk A, B;
        int cA, cB = 0;
        const int rA = locate(K, A.lr, cA);
        const int rB = two ? locate(K + kComputeWarps, B.lr, cB) : rA;
        if (!two) B.lr = A.lr;
        if (!waited && (rA >= wait_at || rB >= wait_at)) {
            if (!wait()) return false;
            waited = true;
        }
        if ((o & 3) == 0) {
            const int K2 = K + kComputeWarps * (lane >> 3);
            int lr2 = 0, c2 = 0;
            if (K2 < total) locate(K2, lr2, c2);
            direction_calls(cx, dcall, K2 < total, lr2, c2, lane);
        }
        load_chunk(cx, dcall, o, cA, lane, A);
        load_chunk(cx, dcall, o + 1, two ? cB : cA, lane, B);
        if (!two) B.valid = false;
        const uint32_t a0 = A.valid ? word_activity(cx.oj, A.cl, A.ca, A.cb, A.ua, A.ub, A.da, A.db, A.d32 & 0xFFFFu) : 0u;
        const uint32_t a1 = A.valid ? word_activity(cx.oj, A.ca, A.cb, A.cq, A.ub, A.uq, A.db, A.dq, A.d32 >> 16) : 0u;
        const uint32_t b0 = B.valid ? word_activity(cx.oj, B.cl, B.ca, B.cb, B.ua, B.ub, B.da, B.db, B.d32 & 0xFFFFu) : 0u;
        const uint32_t b1 = B.valid ? word_activity(cx.oj, B.ca, B.cb, B.cq, B.ub, B.uq, B.db, B.dq, B.d32 >> 16) : 0u;
        push_word<GAME>(cx, q, a0, A.lr, A.wa, A.d32 & 0xFFFFu, lane);
        push_word<GAME>(cx, q, a1, A.lr, A.wa + 1, A.d32 >> 16, lane);
        push_word<GAME>(cx, q, b0, B.lr, B.wa, B.d32 & 0xFFFFu, lane);
        push_word<GAME>(cx, q, b1, B.lr, B.wa + 1, B.d32 >> 16, lane);
    }
    // every warp sees the halo load complete before the step ends, even one without a chunk that
    // reads it: the communication warp reuses the mbarrier, the halo rows and the neighbours'
    // mailbox slot only after the step's barrier, so the load must have landed by then
    if (!waited && !wait()) return false;
    return true;
}

// All remaining active words and sites of the warp. Warp-uniform.
template <int GAME>
__device__ __forceinline__ void flush_rings(const Ctx &cx, Rings &q, int lane) {
    if (q.wt != q.wh) expand_words<GAME>(cx, q, q.wt - q.wh, lane);
    while (q.st != q.sh) drain_sites<GAME, false>(cx, q, min(32u, q.st - q.sh), lane);
}

// Warp-uniform: append each lane's active sites (act: bit t = site t of its class-word, lo_b / hi_b
// the two bits of the sites' direction codes, ebase the class-word's entry base) to the site ring,
// up to 8 per lane and pass (the ring then holds < 32 + 256 entries), updating 32 at a time.
template <int GAME>
__device__ __forceinline__ void push_sites(const Ctx &cx, Rings &q, uint32_t act, uint32_t lo_b, uint32_t hi_b,
                                           uint32_t ebase, int lane) {
    while (__any_sync(0xffffffffu, act != 0u)) {
        const uint32_t cnt = min(static_cast<uint32_t>(__popc(act)), 8u);
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        uint32_t pos = q.st + incl - cnt;
        q.st += __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t k = 0; k < cnt; ++k) {
            const uint32_t t = static_cast<uint32_t>(__ffs(act) - 1);
            act &= act - 1u;
            q.sites[pos & kSiteRingMask] = ebase + (t << 4) + ((lo_b >> t) & 1u) + (((hi_b >> t) & 1u) << 1);
            ++pos;
        }
        while (q.st - q.sh >= 32u) drain_sites<GAME, true>(cx, q, 32u, lane);
    }
}

// The scan of one step on the column-class copy: the class-words of the step's column class in its
// sublattice rows, one per lane (chunks of 32 class-words, ceil(Lq / 32) per row; chunk K of the
// ranges' concatenation to warp K mod 16). A lane draws the Philox call that holds its class-word's
// direction codes (the codes of bit-packed words 4 q .. 4 q + 3: components x, y of call q / 2 for
// an even q, z, w for an odd one), splits them into each site's first and second bit, selects each
// site's drawn neighbour among the east, west, south and north class-words, and pushes the sites
// whose neighbour holds the other strategy. The halo wait as in scan_step. Warp-uniform.
template <int GAME, class Wait>
__device__ __forceinline__ bool scan_step_cls(const Ctx &cx, const Range (&rg)[3], int wait_at, Wait wait, Rings &q,
                                              int warp, int lane) {
    const int Lq = cx.Lq, cpr = cx.cprq, oj = cx.oj;
    const int n0 = rg[0].n * cpr, n1 = rg[1].n * cpr, total = n0 + n1 + rg[2].n * cpr;
    bool waited = wait_at < 0;
    for (int K = warp; K < total; K += kComputeWarps) {
        int r = 0, kk = K;
        if (kk >= n0) {
            kk -= n0;
            r = 1;
            if (kk >= n1) {
                kk -= n1;
                r = 2;
            }
        }
        const int qr = static_cast<int>((static_cast<uint32_t>(kk) * cx.cmagicq) >> 16);
        const int cc = kk - qr * cpr;
        const int lr = (r == 0 ? rg[0].first : r == 1 ? rg[1].first : rg[2].first) + 4 * qr;
        if (!waited && r >= wait_at) {
            if (!wait()) return false;
            waited = true;
        }
        const int qw = 32 * cc + lane;
        const bool valid = qw < Lq;
        const int qq = valid ? qw : 0;
        int i = cx.r0 - cx.H + lr;
        if (i < 0) i += cx.L;
        else if (i >= cx.L) i -= cx.L;
        const uint4 d = philox_rk(
            make_uint4(static_cast<uint32_t>(qq >> 1), static_cast<uint32_t>(i >> 2), cx.kl, cx.kh_dir), *cx.rk);
        const uint32_t ua = unzip32((qq & 1) ? d.z : d.x), ub = unzip32((qq & 1) ? d.w : d.y);
        const uint32_t lo_b = __byte_perm(ua, ub, 0x5410u), hi_b = __byte_perm(ua, ub, 0x7632u);
        const long long rb = static_cast<long long>(lr) * cx.Lw;
        const uint32_t *row = cx.cls + rb;
#define PGG_LDC(OFF) (index_ok(rb + (OFF), cx.n_words, cx.status) ? row[(OFF)] : 0u)
        const uint32_t sx = PGG_LDC(oj * Lq + qq);
        const uint32_t yn = PGG_LDC(oj * Lq + qq - cx.Lw), ys = PGG_LDC(oj * Lq + qq + cx.Lw);
        const uint32_t ye = oj < 3 ? PGG_LDC((oj + 1) * Lq + qq)
                                   : __funnelshift_r(PGG_LDC(qq), PGG_LDC(qq + 1 == Lq ? 0 : qq + 1), 1);
        const uint32_t yw = oj > 0 ? PGG_LDC((oj - 1) * Lq + qq)
                                   : __funnelshift_l(PGG_LDC(3 * Lq + (qq == 0 ? Lq - 1 : qq - 1)), PGG_LDC(3 * Lq + qq), 1);
#undef PGG_LDC
        const uint32_t act = valid ? sx ^ mux(hi_b, mux(lo_b, ye, yw), mux(lo_b, ys, yn)) : 0u;
        push_sites<GAME>(cx, q, act, lo_b, hi_b,
                         static_cast<uint32_t>(lr) << 18 | static_cast<uint32_t>(128 * qq + oj) << 2, lane);
    }
    if (!waited && !wait()) return false;
    return true;
}

// The dense pass: every word of the rows, all 8 sites at once by the shared per-word core
// (pgg_unit.cuh): tasks of tw words of one sublattice row per thread, the 7 x 3 neighbourhood
// slid along the row, one direction call per task. It pays for every word, active or not, and so
// wins over the scan when a large share of the sites can change (early MCS from a random start,
// high cooperator densities).
//
// Task t goes to thread (first + t) mod T, so that a range that follows another starts at the
// threads the previous one left one task short. Returns the number of tasks. tw_set > 0 fixes the
// words per task (a step split into parts sizes them for the whole step).
template <int OJ, int GAME, bool CLS>
__device__ __forceinline__ int dense_rows(const Ctx &cx, const Range &rg, int tid, int first, uint32_t &flips,
                                          int tw_set = 0) {
    if (rg.n <= 0) return 0;
    const int words = rg.n * cx.Lw;
    // words per task: as many as still give every thread of the round a task; a range that starts
    // mid-round (first > 0) sizes its tasks for the threads that round leaves free
    const int free_thr = kComputeThreads - first % kComputeThreads;
    const int tw = tw_set > 0 ? tw_set : words >= 4 * free_thr ? 4 : words >= 2 * free_thr ? 2 : 1;
    const int runs = cx.Lw / tw;  // Lw % 8 == 0, so tasks never straddle a direction call
    const int n_tasks = rg.n * runs;
    const uint32_t kh = static_cast<uint32_t>(cx.k >> 32) | kTagDir;
    int t0 = tid - first % kComputeThreads;
    if (t0 < 0) t0 += kComputeThreads;
    for (int t = t0; t < n_tasks; t += kComputeThreads) {
        const int qr = t / runs;
        const int w0 = (t - qr * runs) * tw;
        const int lr = rg.first + 4 * qr;
        int i = cx.r0 - cx.H + lr;
        if (i < 0) i += cx.L;
        else if (i >= cx.L) i -= cx.L;
        const int wprev = w0 == 0 ? cx.Lw - 1 : w0 - 1;
        uint32_t wl[7], wc[7], wr[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const long long base = static_cast<long long>(lr - 3 + q) * cx.Lw;
            const bool rd = reads_row<GAME>(q);
            wl[q] = rd && index_ok(base + swz(wprev), cx.n_words, cx.status) ? cx.rows[base + swz(wprev)] : 0u;
            wc[q] = rd && index_ok(base + swz(w0), cx.n_words, cx.status) ? cx.rows[base + swz(w0)] : 0u;
        }
        const uint4 dcall = philox_rk(make_uint4(static_cast<uint32_t>(w0 >> 3), static_cast<uint32_t>(i >> 2), cx.kl, kh), *cx.rk);
        UnitCtx u;
        u.k = cx.k;
        u.a = static_cast<uint32_t>(i >> 2);
        u.msk = kNib;
#pragma unroll 1
        for (int w = w0; w < w0 + tw; ++w) {
            const int wn = w + 1 == cx.Lw ? 0 : w + 1;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const long long base = static_cast<long long>(lr - 3 + q) * cx.Lw;
                wr[q] = reads_row<GAME>(q) && index_ok(base + swz(wn), cx.n_words, cx.status) ? cx.rows[base + swz(wn)] : 0u;
            }
            u.gw = w;
            u.d16 = (word_of(dcall, (w >> 1) & 3) >> (16 * (w & 1))) & 0xFFFFu;
            uint32_t sx;
            const uint32_t f = game_flips<OJ, GAME>(wl, wc, wr, u, *cx.rk, cx.table, sx);
            // one thread owns the word in this pass: a plain store (the bits other threads read
            // from it are never among the flipped ones)
            if (f && index_ok(static_cast<long long>(lr) * cx.Lw + swz(w), cx.n_words, cx.status)) {
                cx.rows[lr * cx.Lw + swz(w)] = wc[3] ^ (f << OJ);
                if constexpr (CLS) {
                    // four words share a class-word, each perhaps in another thread's task
                    const long long ci = static_cast<long long>(lr) * cx.Lw + OJ * cx.Lq + (w >> 2);
                    if (index_ok(ci, cx.n_words, cx.status)) atomicXor(&cx.cls[ci], nibble_bits8(f) << (8 * (w & 3)));
                }
            }
            flips += __popc(f);
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                wl[q] = wc[q];
                wc[q] = wr[q];
            }
        }
    }
    return n_tasks;
}

// One step of the dense pass (the rows, the halo wait and the edge hand-over as in step_rows): up to
// three parts through one call site, the halo wait before part `wait_before`, the hand-over after
// part `hand_after`.
template <int OJ, int GAME, bool CLS, class Wait>
__device__ __forceinline__ bool step_dense(const Ctx &cx, int m4, int lo, int hi, int nb, bool split, bool edges,
                                           Wait wait, int tid, uint32_t &flips) {
    constexpr int R = kReadRadius<GAME>;
    const int H = cx.H, in_lo = H + R, in_hi = H + nb - R;
    Range part[3] = {{0, 0}, {0, 0}, {0, 0}};
    int wait_before = -1, hand_after = -1, tw = 0;
    if (edges) {
        // the top and bottom H rows (the whole band if it is thinner than 2H), then the rows between
        // them; words per task for the step as a whole (the edge parts alone would take one each)
        if (nb >= 2 * H) {
            part[0] = srows_in(m4, H, 2 * H);
            part[1] = srows_in(m4, nb, nb + H);
            part[2] = srows_in(m4, 2 * H, nb);
            hand_after = 1;
        } else {
            part[0] = srows_in(m4, H, H + nb);
            hand_after = 0;
        }
        const int all_words = srows_in(m4, H, H + nb).n * cx.Lw;
        tw = all_words >= 4 * kComputeThreads ? 4 : all_words >= 2 * kComputeThreads ? 2 : 1;
    } else if (!split) {
        part[0] = srows_in(m4, lo, hi);
    } else if (in_hi > in_lo) {
        part[0] = srows_in(m4, in_lo, in_hi);
        part[1] = srows_in(m4, lo, in_lo);
        part[2] = srows_in(m4, in_hi, hi);
        wait_before = 1;
    } else {
        part[0] = srows_in(m4, lo, hi);
        wait_before = 0;
    }
    int next = 0;
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        if (k == wait_before && !wait()) return false;
        next += dense_rows<OJ, GAME, CLS>(cx, part[k], tid, next, flips, tw);
        if (k == hand_after) {
            fence_async_shared();  // the edge rows' writes, for the bulk store
            edges_arrive();
        }
    }
    return true;
}

// One step: with `split`, first the rows whose reads stay inside the band, then -- once the
// halo has landed -- the rest; then every remaining active site. With `edges` (the last step of a
// block of s > 1 steps, band rows only, no halo wait), first the band's top and bottom H rows,
// which the exchange warp publishes as soon as every compute thread has handed them over, then
// the rows between them.
template <int GAME, bool CLS, class Wait>
__device__ __forceinline__ bool step_rows(const Ctx &cx, int m4, int lo, int hi, int nb, bool split, bool edges,
                                          Wait wait, Rings &q, int warp, int lane) {
    constexpr int R = kReadRadius<GAME>;
    Range rg[3] = {{0, 0}, {0, 0}, {0, 0}};
    int wait_at = -1;
    // rows [in_lo, in_hi) read band rows only; lo <= H < in_lo and in_hi <= H + nb <= hi
    const int in_lo = cx.H + R, in_hi = cx.H + nb - R;
    Range interior{0, 0};  // with `edges`: the rows of the second phase
    if (edges) {
        const int H = cx.H;
        if (nb >= 2 * H) {
            rg[0] = srows_in(m4, H, 2 * H);
            rg[1] = srows_in(m4, nb, nb + H);
            interior = srows_in(m4, 2 * H, nb);
        } else {
            rg[0] = srows_in(m4, H, H + nb);
        }
    } else if (!split) {
        rg[0] = srows_in(m4, lo, hi);
    } else if (in_hi <= in_lo) {  // a band too thin for an interior
        rg[0] = srows_in(m4, lo, hi);
        wait_at = 0;
    } else {
        rg[0] = srows_in(m4, in_lo, in_hi);
        rg[1] = srows_in(m4, lo, in_lo);
        rg[2] = srows_in(m4, in_hi, hi);
        wait_at = 1;
    }
#pragma unroll 1
    for (int phase = 0; phase < (edges ? 2 : 1); ++phase) {
        if (phase == 1) {  // the edge rows are done: hand them over, then the rows between them
            fence_async_shared();
            edges_arrive();
            rg[0] = interior;
            rg[1] = Range{0, 0};
        }
        if constexpr (CLS) {
            if (!scan_step_cls<GAME>(cx, rg, wait_at, wait, q, warp, lane)) return false;
            while (q.st != q.sh) drain_sites<GAME, true>(cx, q, min(32u, q.st - q.sh), lane);
        } else {
            if (!scan_step<GAME>(cx, rg, wait_at, wait, q, warp, lane)) return false;
            flush_rings<GAME>(cx, q, lane);
        }
    }
    return true;
}

// --- TMA bulk copies and the CTA's mbarrier (PTX) ------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// global -> shared, completion counted in bytes on the mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// shared -> global in the thread's bulk async-group
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit_and_wait() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// 4-byte global -> shared copy in the thread's cp.async group, and the wait for all of them
__device__ __forceinline__ void copy_async4(uint32_t *dst, const uint32_t *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// 16-byte global -> shared copy (both 16-byte aligned) in the thread's cp.async group
__device__ __forceinline__ void copy_async16(uint32_t *dst, const uint32_t *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void copy_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}


// Barrier of the compute warps only (the communication warp does not take part).
__device__ __forceinline__ void compute_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(kComputeThreads) : "memory"); }

// try_wait calls a compute warp makes on the halo mbarrier before it gives up (each call may
// suspend the thread for a short time; a bulk copy from L2 lands within microseconds).
constexpr unsigned int kMbarTries = 1u << 26;

// CLS: keep the column-class copy of the rows and scan it (shared memory for both copies).
template <int GAME, bool CLS>
__global__ void __launch_bounds__(kResThreads, 1) k_resident(const __grid_constant__ ResidentParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    constexpr int R = kReadRadius<GAME>;
    const int L = p.L, Lw = p.Lw, S = p.s, H = p.H;
    const int b = blockIdx.x, nbnd = p.n_bands;
    const int r0 = band_start(b, L, nbnd), nb = band_start(b + 1, L, nbnd) - r0;
    const int nb_max = (L + nbnd - 1) / nbnd;
    uint32_t *s_table = smem;
    const size_t rows_words = static_cast<size_t>(nb_max + 2 * H) * Lw;
    uint32_t *s_rows = smem + kTableEntries;                 // (nb_max + 2H) rows
    uint32_t *s_cls = s_rows + rows_words;                   // their class copy (CLS)
    uint2 *s_wring = reinterpret_cast<uint2 *>(s_cls + (CLS ? rows_words : 0));
    uint32_t *s_sring = reinterpret_cast<uint32_t *>(s_wring + kComputeWarps * kWordRingCap);
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ volatile int s_abort;
    __shared__ unsigned long long s_warp[kComputeWarps];
    __shared__ unsigned int s_flips[3];  // adoptions in the CTA's steps j (mod 3)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool comm = tid >= kComputeThreads;  // the last warp exchanges halos, the others compute
    const int up = (b + nbnd - 1) % nbnd, down = (b + 1) % nbnd;
    const size_t edge = static_cast<size_t>(H) * Lw;                  // words of H rows
    const size_t slot = CLS ? 2 * edge : edge;                        // a mailbox side: rows (+ class copy)
    const uint32_t edge_bytes = static_cast<uint32_t>(edge * sizeof(uint32_t));
    const PhiloxKeys &rk = p.rk;  // read from the parameter space: constant operands
    // bulk copies need 16-byte aligned rows (the same answer in every CTA: all stop together)
    if ((smem_u32(s_rows) & 15u) != 0u || (smem_u32(s_cls) & 15u) != 0u ||
        (reinterpret_cast<uintptr_t>(p.mailbox) & 15u) != 0u || (reinterpret_cast<uintptr_t>(p.lat8) & 15u) != 0u) {
        if (tid == 0) atomicOr(p.status, 2);
        return;
    }
    for (int t = tid; t < kTableEntries; t += kResThreads) copy_async4(&s_table[t], &p.table[t]);
    if (tid == 0) {
        s_abort = 0;
        mbar_init(&s_mbar, 1);
        // the step before the first one: the adoptions the band saw in the last step of the
        // previous launch (a hint for the first pass; it never affects results)
        s_flips[2] = p.hint ? p.hint[b] : 0u;
        s_flips[0] = 0u;
        s_flips[1] = 0u;
    }
    // stage band + halo (rows r0 - H .. r0 + nb + H - 1, periodic) with 4-byte asynchronous
    // copies (cp.async: many loads in flight per thread, each word to its place); thread t
    // copies column t mod Lw of every (T / Lw)-th row, so a copy costs a few adds
    const int n_local = nb + 2 * H;
    const int rows_per_pass = kResThreads / Lw;   // >= 1: a resident row has at most 448 words
    const int col = tid % Lw, row_first = tid / Lw;
    const int scol = swz(col);
    if (row_first < rows_per_pass) {
        int g = wrap_small(r0 - H + row_first, L);
        if (p.lat8) {
            // uint8 lattice: the word's 32 bytes in two 16-byte loads (rows start 256-byte aligned)
#pragma unroll 4
            for (int lr = row_first; lr < n_local; lr += rows_per_pass) {
                const size_t off = static_cast<size_t>(g) * L + 32 * static_cast<size_t>(col);
                if (index_ok(static_cast<long long>(off) + 31, static_cast<long long>(L) * L, p.status)) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(p.lat8 + off);
                    s_rows[lr * Lw + scol] = pack_bytes32(src[0], src[1]);
                }
                g += rows_per_pass;
                if (g >= L) g -= L;
            }
        } else {
            for (int lr = row_first; lr < n_local; lr += rows_per_pass) {
                if (index_ok(static_cast<long long>(g) * Lw + col, static_cast<long long>(L) * Lw, p.status))
                    copy_async4(&s_rows[lr * Lw + scol], &p.lat[static_cast<size_t>(g) * Lw + col]);
                g += rows_per_pass;
                if (g >= L) g -= L;
            }
        }
    }
    // the class copy: staged from the lattice's copy in global memory when it holds this lattice
    // (16-byte copies, its rows are not swizzled), else built from the rows once they have landed
    const int q16 = Lw >> 2;  // 16-byte chunks of a row
    if (CLS && p.cls_load && p.cls_g && tid / q16 < kResThreads / q16) {
        const int cc = tid % q16, rows_per_pass16 = kResThreads / q16;
        int g = wrap_small(r0 - H + tid / q16, L);
        for (int lr = tid / q16; lr < n_local; lr += rows_per_pass16) {
            if (index_ok(static_cast<long long>(lr) * Lw + 4 * cc + 3, static_cast<long long>(n_local) * Lw, p.status) &&
                index_ok(static_cast<long long>(g) * Lw + 4 * cc + 3, static_cast<long long>(L) * Lw, p.status))
                copy_async16(&s_cls[lr * Lw + 4 * cc], &p.cls_g[static_cast<size_t>(g) * Lw + 4 * cc]);
            g += rows_per_pass16;
            if (g >= L) g -= L;
        }
    }
    copy_async_wait_all();
    fence_async_shared();  // the staged halo rows are later overwritten by bulk loads
    __syncthreads();
    if constexpr (CLS) {
        if (!(p.cls_load && p.cls_g)) {
            build_class_rows(s_rows, s_cls, n_local, Lw, tid, kResThreads, p.status);
            fence_async_shared();  // and so are the class copy's
            __syncthreads();
        }
    }

    Ctx cx;
    cx.rows = s_rows;
    cx.cls = s_cls;
    cx.Lq = Lw >> 2;
    cx.cprq = (cx.Lq + 31) >> 5;
    cx.cmagicq = (65536u + static_cast<uint32_t>(cx.cprq) - 1u) / static_cast<uint32_t>(cx.cprq);
    cx.table = s_table;
    cx.L = L;
    cx.Lw = Lw;
    cx.r0 = r0;
    cx.H = H;
    cx.rk = &rk;
    cx.cpr = (Lw + 63) >> 6;
    cx.cmagic = (65536u + static_cast<uint32_t>(cx.cpr) - 1u) / static_cast<uint32_t>(cx.cpr);
    cx.n_words = static_cast<long long>(n_local) * Lw;
    cx.status = p.status;
    Rings q;
    q.words = s_wring + (warp < kComputeWarps ? warp : 0) * kWordRingCap;
    q.sites = s_sring + (warp < kComputeWarps ? warp : 0) * kSiteRingCap;
    q.wh = q.wt = q.sh = q.st = 0;
    // the dense pass takes a step when the previous step flipped more than this many sites of the
    // band (a share of the sites one step updates)
    const unsigned int dense_above =
        static_cast<unsigned int>((static_cast<unsigned long long>(nb) * L / 16) * p.dense_per_mille / 1000);
    uint4 ocall = make_uint4(0, 0, 0, 0);
    uint64_t ocall_idx = ~0ull;
    const int n_blocks = 16 * p.n_mcs / S;
    bool load_pending = false;  // communication lane: a halo load not yet seen complete
    // publish the band's top and bottom H rows (and their class copy) after block blk for the
    // neighbours' next block: bulk stores straight from the rows, complete before the counter is
    // released (and before the issuer reaches the step's barrier, after which they change again)
    auto publish = [&](int blk) {
        uint32_t *to_top = p.mailbox + ((static_cast<size_t>(b) * 2 + (blk & 1)) * 2 + 0) * slot;
        uint32_t *to_bot = p.mailbox + ((static_cast<size_t>(b) * 2 + (blk & 1)) * 2 + 1) * slot;
        bulk_store(to_top, s_rows + static_cast<size_t>(H) * Lw, edge_bytes);
        bulk_store(to_bot, s_rows + static_cast<size_t>(nb) * Lw, edge_bytes);
        if (CLS) {
            bulk_store(to_top + edge, s_cls + static_cast<size_t>(H) * Lw, edge_bytes);
            bulk_store(to_bot + edge, s_cls + static_cast<size_t>(nb) * Lw, edge_bytes);
        }
        bulk_commit_and_wait();
        fence_async_global();
        __threadfence();
        store_release(&p.ctr[b], p.ctr_base + static_cast<unsigned int>(blk + 1));
    };
    for (int blk = 0; blk < n_blocks; ++blk) {
        for (int jb = 0; jb < S; ++jb) {
            const int j = blk * S + jb;
            const uint64_t k = p.k0 + static_cast<uint64_t>(j);
            const bool fresh_halo = jb == 0 && blk > 0;  // the halo is being refreshed for this step
            const bool edges = S > 1 && jb == S - 1;      // the edge rows go out mid-step
            if (comm) {
                // fetch the neighbours' rows after block blk - 1 into the halo, asynchronously
                if (tid == kComputeThreads && fresh_halo) {
                    unsigned int it = 0;
                    const unsigned int want = p.ctr_base + static_cast<unsigned int>(blk);
                    while ((load_acquire(&p.ctr[up]) < want || load_acquire(&p.ctr[down]) < want) && it < p.spin_limit) {
                        __nanosleep(32);
                        ++it;
                    }
                    if (it >= p.spin_limit) {
                        atomicOr(p.status, 1);
                        s_abort = 1;
                    } else {
                        const int par = (blk - 1) & 1;
                        const uint32_t *from_up = p.mailbox + ((static_cast<size_t>(up) * 2 + par) * 2 + 1) * slot;
                        const uint32_t *from_down = p.mailbox + ((static_cast<size_t>(down) * 2 + par) * 2 + 0) * slot;
                        fence_async_global();  // the acquired rows, for the async proxy's reads
                        mbar_expect_tx(&s_mbar, (CLS ? 4 : 2) * edge_bytes);
                        bulk_load(s_rows, from_up, edge_bytes, &s_mbar);
                        bulk_load(s_rows + static_cast<size_t>(nb + H) * Lw, from_down, edge_bytes, &s_mbar);
                        if (CLS) {
                            bulk_load(s_cls, from_up + edge, edge_bytes, &s_mbar);
                            bulk_load(s_cls + static_cast<size_t>(nb + H) * Lw, from_down + edge, edge_bytes, &s_mbar);
                        }
                        load_pending = true;
                    }
                }
                if (edges) {
                    // the last step of a block with s > 1: its rows are band rows only and read no
                    // halo; the compute warps update the top and bottom H rows first and hand them
                    // over, and they go out while the rows between them are updated
                    edges_wait();
                    if (tid == kComputeThreads) publish(blk);
                }
                __syncwarp();
            } else {
                if ((k >> 5) != ocall_idx) {
                    ocall_idx = k >> 5;
                    ocall = philox_rk(make_uint4(static_cast<uint32_t>(ocall_idx), static_cast<uint32_t>(ocall_idx >> 32), 0u,
                                                 kTagOffset), rk);
                }
                const int o = static_cast<int>((word_of(ocall, static_cast<int>((k >> 3) & 3)) >> (4 * (k & 7))) & 15u);
                cx.kl = static_cast<uint32_t>(k);
                cx.k = k;
                cx.oj = o & 3;
                cx.kh_dir = static_cast<uint32_t>(k >> 32) | kTagDir;
                cx.kh_u = static_cast<uint32_t>(k >> 32) | kTagU;
                // local row lr is global row r0 - H + lr: a sublattice row iff lr = oi - r0 + H (mod 4)
                const int m4 = ((o >> 2) - r0 + H) & 3;
                const int e = R * (S - 1 - jb);  // halo rows updated on each side in this step
                const int lo = H - e, hi = H + nb + e;
                const int parity = (blk - 1) & 1;
                auto wait = [&]() -> bool {
                    unsigned int it = 0;
                    while (!mbar_try_wait(&s_mbar, static_cast<uint32_t>(parity))) {
                        if (s_abort || ++it >= kMbarTries) return false;
                    }
                    return true;
                };
                if (tid == 0) s_flips[(j + 1) % 3] = 0u;  // the slot of step j + 1 (last read in step j - 1)
                const bool dense = s_flips[(j + 2) % 3] > dense_above;  // the previous step's adoptions
                q.flips = 0;
                bool ok = true;
                if (dense) {
                    switch (o & 3) {
                        case 0: ok = step_dense<0, GAME, CLS>(cx, m4, lo, hi, nb, fresh_halo, edges, wait, tid, q.flips); break;
                        case 1: ok = step_dense<1, GAME, CLS>(cx, m4, lo, hi, nb, fresh_halo, edges, wait, tid, q.flips); break;
                        case 2: ok = step_dense<2, GAME, CLS>(cx, m4, lo, hi, nb, fresh_halo, edges, wait, tid, q.flips); break;
                        default: ok = step_dense<3, GAME, CLS>(cx, m4, lo, hi, nb, fresh_halo, edges, wait, tid, q.flips); break;
                    }
                } else {
                    ok = step_rows<GAME, CLS>(cx, m4, lo, hi, nb, fresh_halo, edges, wait, q, warp, lane);
                }
                // the step's adoptions, for the next step's choice of pass
                const unsigned int wf = __reduce_add_sync(0xffffffffu, q.flips);
                if (lane == 0 && wf) atomicAdd(&s_flips[j % 3], wf);
                if (!ok) {
                    s_abort = 1;
                    q.wh = q.wt;  // the step is abandoned
                    q.sh = q.st;
                }
                __syncwarp();
                fence_async_shared();  // this thread's lattice writes, for the bulk store below
            }
            __syncthreads();
            if (s_abort) {
                // a wait ran out: make sure no bulk copy still targets this CTA's shared memory,
                // then stop; the lattice in global memory is left as it was
                if (tid == kComputeThreads && load_pending) {
                    unsigned int it = 0;
                    while (!mbar_try_wait(&s_mbar, static_cast<uint32_t>((blk - 1) & 1)) && ++it < kMbarTries) {
                    }
                    // the halo load was never seen to land: the CTA leaves with a copy into its
                    // shared memory possibly in flight, which the host must treat as fatal
                    if (it >= kMbarTries) atomicOr(p.status, 8);
                }
                return;
            }
            if (fresh_halo) load_pending = false;
            if (S == 1) {
                // one step per block: the rows go out after the step (the next step updates them only
                // after its halo wait, which follows this copy's completion)
                if (tid == kComputeThreads) publish(blk);
                __syncwarp();
            }
            if (!comm && (j & 15) == 15 && p.counts) {
                unsigned long long c = 0;
                for (int x = tid; x < nb * Lw; x += kComputeThreads) c += __popc(s_rows[H * Lw + x]);
#pragma unroll
                for (int sft = 16; sft > 0; sft >>= 1) c += __shfl_down_sync(0xffffffffu, c, sft);
                if (lane == 0) s_warp[warp] = c;
                compute_barrier();
                if (tid == 0) {
                    unsigned long long tot = 0;
                    for (int w = 0; w < kComputeWarps; ++w) tot += s_warp[w];
                    // MCS m's bands add into slot m mod kResidentCountSlots; the last band to add
                    // writes the count and clears the slot. A band in block k has waited for its
                    // neighbours to finish block k - 1, so every band has finished block
                    // k - n_bands / 2: no band reaches a slot again before it is clear (the launch
                    // checks the slots cover that lag), and every slot is clear when the launch ends.
                    const int m = j >> 4, slot = m % kResidentCountSlots;
                    atomicAdd(&p.count_acc[slot], tot);
                    __threadfence();
                    if (atomicAdd(&p.count_tick[slot], 1u) == static_cast<unsigned int>(nbnd) - 1u) {
                        __threadfence();
                        p.counts[m] = atomicExch(&p.count_acc[slot], 0ull);
                        atomicExch(&p.count_tick[slot], 0u);
                    }
                }
            }
        }
    }
    __syncthreads();  // the last bulk store has completed (its issuer waited) before the band is stored
    if (tid == 0 && p.hint) p.hint[b] = s_flips[(16 * p.n_mcs - 1) % 3];
    // the band's class copy, for the next launch on this lattice
    if (CLS && p.cls_g) {
        for (int x = tid; x < nb * q16; x += kResThreads) {
            const int lr = x / q16, cc = x - lr * q16;
            if (index_ok(static_cast<long long>(r0 + lr) * Lw + 4 * cc + 3, static_cast<long long>(L) * Lw, p.status))
                *reinterpret_cast<uint4 *>(&p.cls_g[static_cast<size_t>(r0 + lr) * Lw + 4 * cc]) =
                    *reinterpret_cast<const uint4 *>(&s_cls[(lr + H) * Lw + 4 * cc]);
        }
    }
    // store the band (the same column-per-thread walk)
    if (row_first < rows_per_pass) {
        if (p.lat8) {
            for (int lr = row_first; lr < nb; lr += rows_per_pass) {
                const size_t off = static_cast<size_t>(r0 + lr) * L + 32 * static_cast<size_t>(col);
                if (index_ok(static_cast<long long>(off) + 31, static_cast<long long>(L) * L, p.status)) {
                    const uint32_t w = s_rows[(lr + H) * Lw + scol];
                    uint4 *dst = reinterpret_cast<uint4 *>(p.lat8 + off);
                    dst[0] = unpack_bits16(w & 0xFFFFu);
                    dst[1] = unpack_bits16(w >> 16);
                }
            }
        } else {
            for (int lr = row_first; lr < nb; lr += rows_per_pass) {
                if (index_ok(static_cast<long long>(r0 + lr) * Lw + col, static_cast<long long>(L) * Lw, p.status))
                    p.lat[static_cast<size_t>(r0 + lr) * Lw + col] = s_rows[(lr + H) * Lw + scol];
            }
        }
    }
}

// Shared memory of a launch: table, band + halo rows (twice with the column-class copy, cls), the
// warps' rings.
size_t resident_smem_bytes(int L, int n_bands, int game, int s, bool cls) {
    const int H = kReadRadius<kGroupGame> * s;  // the group game's halo bounds the pairwise game's
    (void)game;
    const size_t Lw = static_cast<size_t>(L / 32);
    const size_t max_rows = static_cast<size_t>((L + n_bands - 1) / n_bands);
    const size_t copies = cls ? 2 : 1;
    return sizeof(uint32_t) * (kTableEntries + copies * (max_rows + 2 * H) * Lw) +
           static_cast<size_t>(kComputeWarps) * (kWordRingCap * sizeof(uint2) + kSiteRingCap * sizeof(uint32_t));
}

}  // namespace

// Bands for a lattice of side L: one per SM when every band keeps at least 3 rows (the rows a
// block of one step publishes must be band rows) and its rows fit the shared memory with one
// step per exchange; 0 when the lattice cannot be resident.
int resident_bands(int layout, int L, int sms, size_t smem_optin) {
    (void)layout;
    if (L < 256 || L % 256 != 0 || sms < 1) return 0;
    int n = sms;
    while (n > 1 && L / n < kReadRadius<kGroupGame>) --n;
    const int max_rows = (L + n - 1) / n;
    return resident_smem_bytes(L, n, kGroupGame, 1, false) <= smem_optin && max_rows + 6 <= kMaxLocalRows && L / 32 <= kMaxRowWords
               ? n
               : 0;
}

// Largest s in {4, 2, 1} (sublattice steps per halo exchange) whose rows fit the shared memory.
int resident_max_steps_per_exchange(int L, int n_bands, size_t smem_optin) {
    const int max_rows = (L + n_bands - 1) / n_bands;
    for (int s = kMaxStepsPerExchange; s > 1; s >>= 1)
        if (resident_smem_bytes(L, n_bands, kGroupGame, s, false) <= smem_optin && L / n_bands >= 3 * s &&
            max_rows + 6 * s <= kMaxLocalRows)
            return s;
    return 1;
}

// Whether a launch with s steps per exchange fits the column-class copy beside the rows.
bool resident_class_copy(int L, int n_bands, int s, size_t smem_optin) {
    return L % 128 == 0 && resident_smem_bytes(L, n_bands, kGroupGame, s, true) <= smem_optin;
}

// [band][parity][top, bottom][rows, class copy][H rows][Lw]
size_t resident_mailbox_words(int L, int n_bands) { return static_cast<size_t>(n_bands) * 2 * 2 * 2 * kMaxHalo * (L / 32); }

cudaError_t launch_resident(const ResidentArgs &a, cudaStream_t s) {
    if (a.n_bands < 1 || a.L % 256 != 0) return cudaErrorInvalidValue;
    if (a.steps_per_exchange != 1 && a.steps_per_exchange != 2 && a.steps_per_exchange != 4) return cudaErrorInvalidValue;
    ResidentParams p;
    p.lat = a.lat;
    p.lat8 = a.lat8;
    p.L = a.L;
    p.Lw = a.L / 32;
    p.n_bands = a.n_bands;
    p.s = a.steps_per_exchange;
    p.H = (a.game == kPairGame ? kReadRadius<kPairGame> : kReadRadius<kGroupGame>) * p.s;
    if (a.L / a.n_bands < p.H) return cudaErrorInvalidValue;  // published rows must be band rows
    // a band runs at most n_bands / 2 + 1 halo blocks ahead of any other: the count slots must
    // cover that many MCS (152 bands, 4 steps per block: 20 of 64)
    if ((a.n_bands / 2 + 2) * p.s > 16 * kResidentCountSlots) return cudaErrorInvalidValue;
    if ((a.L + a.n_bands - 1) / a.n_bands + 2 * p.H > kMaxLocalRows || p.Lw > kMaxRowWords) return cudaErrorInvalidValue;
    p.seed = a.seed;
    p.k0 = a.k0;
    p.n_mcs = a.n_mcs;
    p.table = a.table;
    p.mailbox = a.mailbox;
    p.ctr = a.ctr;
    p.ctr_base = a.ctr_base;
    p.counts = a.counts;
    p.count_acc = a.count_acc;
    p.count_tick = a.count_tick;
    if (a.counts && (!a.count_acc || !a.count_tick)) return cudaErrorInvalidValue;
    p.status = a.status;
    p.spin_limit = a.spin_limit;
    p.hint = a.hint;
    p.dense_per_mille = a.dense_per_mille;
    p.cls_g = a.class_copy ? a.cls_g : nullptr;
    p.cls_load = a.class_copy && a.cls_g && a.cls_load ? 1 : 0;
    p.rk = philox_round_keys(a.seed);
    const bool cls = a.class_copy;
    const size_t smem = resident_smem_bytes(a.L, a.n_bands, a.game, p.s, cls);
    const void *kernel = a.game == kPairGame
                             ? (cls ? reinterpret_cast<const void *>(k_resident<kPairGame, true>)
                                    : reinterpret_cast<const void *>(k_resident<kPairGame, false>))
                             : (cls ? reinterpret_cast<const void *>(k_resident<kGroupGame, true>)
                                    : reinterpret_cast<const void *>(k_resident<kGroupGame, false>));
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (a.reset_ctr) {
        e = cudaMemsetAsync(a.ctr, 0, sizeof(unsigned int) * a.n_bands, s);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {&p};
    return cudaLaunchCooperativeKernel(kernel, dim3(a.n_bands), dim3(kResThreads), args, smem, s);
}

}  // namespace pgg
