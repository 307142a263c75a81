// pgg_device.cuh -- device-side building blocks shared by the lattice kernels:
// the Philox4x32-10 generator and the draws of the random-stream contract declared in
// include/pgg.h, periodic indexing, and the strategy-count stencil.
#pragma once

#include <cstdint>

namespace pgg {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// products whose high halves are mixed into the other counter words with the key;
// the key advances by two Weyl increments between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Stream tags, bits 24..31 of counter word 3.
constexpr uint32_t kTagInit = 1u << 24;
constexpr uint32_t kTagOffset = 2u << 24;
constexpr uint32_t kTagDir = 3u << 24;
constexpr uint32_t kTagU = 4u << 24;

// Group-count sums S lie in [0, 25]; thresholds are indexed (s_x*26 + S_x)*26 + S_y.
constexpr int kSRange = 26;
constexpr int kTableEntries = 2 * kSRange * kSRange;
// Pairwise game (Section VI): the table is indexed (s_x*5 + n_x)*5 + n_y, n = cooperating
// neighbours (0..4); it uses the first kPairEntries words of the same buffer.
constexpr int kNRange = 5;
constexpr int kPairEntries = 2 * kNRange * kNRange;

// Games the step kernels play: the public goods game in groups (Section III) and the
// pairwise matrix game (Section VI). kReadRadius: rows / columns an update reads on each
// side of its site.
enum Game { kGroupGame = 0, kPairGame = 1 };
template <int GAME>
constexpr int kReadRadius = GAME == kPairGame ? 2 : 3;

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                        uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c0;
        const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c2;
        const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ k1;
        c1 = static_cast<uint32_t>(p1);
        c3 = static_cast<uint32_t>(p0);
        c0 = n0;
        c2 = n2;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Round keys of Philox4x32-10 for one seed: round r uses (k0 + r W0, k1 + r W1). Built once
// on the host and passed in kernel parameters, so that every round reads its key as a
// constant operand instead of recomputing it.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

inline PhiloxKeys philox_round_keys(uint64_t seed) {
    PhiloxKeys rk;
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = k0;
        rk.k1[r] = k1;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return rk;
}

__device__ __forceinline__ void philox_round(uint4 &c, uint32_t k0, uint32_t k1) {
    const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c.x;
    const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c.z;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ k0, static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ k1, static_cast<uint32_t>(p0));
}

// Philox4x32-10 with precomputed round keys.
__device__ __forceinline__ uint4 philox_rk(uint4 c, const PhiloxKeys &rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) philox_round(c, rk.k0[r], rk.k1[r]);
    return c;
}

// Two independent counters, rounds interleaved for instruction-level parallelism.
__device__ __forceinline__ void philox_rk2(uint4 &a, uint4 &b, const PhiloxKeys &rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(a, rk.k0[r], rk.k1[r]);
        philox_round(b, rk.k0[r], rk.k1[r]);
    }
}

__device__ __forceinline__ uint32_t word_of(const uint4 &w, int idx) {
    return idx == 0 ? w.x : idx == 1 ? w.y : idx == 2 ? w.z : w.w;
}

// Sublattice offset of step k, 0..15 (row offset o >> 2, column offset o & 3).
__device__ __forceinline__ int draw_offset(uint64_t seed, uint64_t k) {
    const uint64_t m = k >> 5;
    const uint4 w = philox4x32_10(static_cast<uint32_t>(m), static_cast<uint32_t>(m >> 32), 0u,
                                  kTagOffset, static_cast<uint32_t>(seed),
                                  static_cast<uint32_t>(seed >> 32));
    return static_cast<int>((word_of(w, static_cast<int>((k >> 3) & 3)) >> (4 * (k & 7))) & 15u);
}

// The 32-bit word holding the direction codes of sublattice sites b with the same b >> 4
// in sublattice row a at step k (2 bits per site, site b at bits 2 (b & 15)).
__device__ __forceinline__ uint32_t draw_dir_word(uint64_t seed, uint64_t k, uint32_t a,
                                                  uint32_t b) {
    const uint4 w = philox4x32_10(b >> 6, a, static_cast<uint32_t>(k),
                                  static_cast<uint32_t>(k >> 32) | kTagDir,
                                  static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    return word_of(w, static_cast<int>((b >> 4) & 3));
}

// The four adoption draws of sublattice sites 4g..4g+3 of sublattice row a at step k.
__device__ __forceinline__ uint4 draw_u4(uint64_t seed, uint64_t k, uint32_t a, uint32_t g) {
    return philox4x32_10(g, a, static_cast<uint32_t>(k), static_cast<uint32_t>(k >> 32) | kTagU,
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// Periodic wrap of a coordinate at most L away from [0, L).
__device__ __forceinline__ int wrap_near(int v, int L) {
    return v < 0 ? v + L : (v >= L ? v - L : v);
}

// Initial condition (Section III) of bit-packed word wi (sites 32 wi .. 32 wi + 31, row-major
// index): one Philox call per 4 sites, site C iff its word is below thr = floor(p 2^32).
__device__ __forceinline__ uint32_t init_packed_word(uint64_t wi, uint64_t seed, uint64_t thr) {
    uint32_t bits = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint64_t q = wi * 8 + c;
        const uint4 w = philox4x32_10(static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32), 0u, kTagInit,
                                      static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
        bits |= (static_cast<uint32_t>(static_cast<uint64_t>(w.x) < thr) << (4 * c + 0)) |
                (static_cast<uint32_t>(static_cast<uint64_t>(w.y) < thr) << (4 * c + 1)) |
                (static_cast<uint32_t>(static_cast<uint64_t>(w.z) < thr) << (4 * c + 2)) |
                (static_cast<uint32_t>(static_cast<uint64_t>(w.w) < thr) << (4 * c + 3));
    }
    return bits;
}

// Checked build (compiled with -DPGG_CHECKED=1, a separate library used by the tests): every
// shared- and global-memory index of the step kernels is tested against its buffer before the
// access; a failed test sets bit 2 (value 4) of the context's status word and skips the access,
// so the host reports it at the next synchronising call. In the normal build the test is the
// constant true and costs nothing.
#ifndef PGG_CHECKED
#define PGG_CHECKED 0
#endif
constexpr int kStatusIndexCheck = 4;

__device__ __forceinline__ bool index_ok(long long idx, long long n, int *status) {
#if PGG_CHECKED
    if (idx >= 0 && idx < n) return true;
    if (status) atomicOr(status, kStatusIndexCheck);
    return false;
#else
    (void)idx;
    (void)n;
    (void)status;
    return true;
#endif
}

}  // namespace pgg
