// pgg_kernels_basic.cu -- initial condition, cooperator count, layout conversion and the
// per-site baseline step kernel.
//
// The baseline kernel is the plain statement of one sublattice step on the GPU: one
// thread per 8 consecutive sublattice sites of a sublattice row, operands read from
// global memory with the periodic wrap, group counts by the 13-site stencil
// S(z) = 5 s_z + 2 (4 nearest) + 2 (4 diagonal) + (4 at distance 2), which is the sum of
// the cooperator counts of the five groups of z (Section III, Fig. 1); for the pairwise
// game (Section VI) the count of cooperating nearest neighbours instead.
#include <cuda_runtime.h>

#include "pgg_device.cuh"
#include "pgg_internal.h"

namespace pgg {
namespace {

// ---------------------------------------------------------------------------------
// Initial condition (Section III): site C with probability p. One Philox call gives
// the four sites 4q .. 4q+3 (row-major index).
// ---------------------------------------------------------------------------------
__global__ void k_init_u8(uint8_t *__restrict__ lat, uint64_t n_quads, uint64_t seed,
                          uint64_t thr) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n_quads;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 w = philox4x32_10(static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32),
                                      0u, kTagInit, static_cast<uint32_t>(seed),
                                      static_cast<uint32_t>(seed >> 32));
        uchar4 v;
        v.x = static_cast<uint64_t>(w.x) < thr;
        v.y = static_cast<uint64_t>(w.y) < thr;
        v.z = static_cast<uint64_t>(w.z) < thr;
        v.w = static_cast<uint64_t>(w.w) < thr;
        reinterpret_cast<uchar4 *>(lat)[q] = v;
    }
}

__global__ void k_init_packed(uint32_t *__restrict__ lat, uint64_t n_words, uint64_t seed,
                              uint64_t thr) {
    for (uint64_t wi = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; wi < n_words;
         wi += (uint64_t)gridDim.x * blockDim.x)
        lat[wi] = init_packed_word(wi, seed, thr);
}

// ---------------------------------------------------------------------------------
// Counting (numerator of Eq. (4)): population count of the buffer.
// ---------------------------------------------------------------------------------
__global__ void k_popcount(const uint4 *__restrict__ p, uint64_t n_vec, unsigned long long *out) {
    unsigned long long acc = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n_vec;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 w = p[v];
        acc += __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ unsigned long long warp_sum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_sum[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (blockDim.x >> 5) ? warp_sum[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0 && acc) atomicAdd(out, acc);
    }
}

// ---------------------------------------------------------------------------------
// Layout conversion.
// ---------------------------------------------------------------------------------
__global__ void k_pack(const uint8_t *__restrict__ src, uint32_t *__restrict__ dst,
                       uint64_t n_words) {
    for (uint64_t wi = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; wi < n_words;
         wi += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 *s = reinterpret_cast<const uint4 *>(src + wi * 32);
        uint32_t bits = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 v = s[h];
            const uint32_t parts[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int byte = 0; byte < 4; ++byte)
                    bits |= static_cast<uint32_t>(((parts[q] >> (8 * byte)) & 0xffu) != 0)
                            << (16 * h + 4 * q + byte);
        }
        dst[wi] = bits;
    }
}

__global__ void k_unpack(const uint32_t *__restrict__ src, uint8_t *__restrict__ dst,
                         uint64_t n_words) {
    for (uint64_t wi = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; wi < n_words;
         wi += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t bits = src[wi];
        uint4 *d = reinterpret_cast<uint4 *>(dst + wi * 32);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t parts[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t nib = (bits >> (16 * h + 4 * q)) & 0xfu;
                parts[q] = (nib & 1u) | ((nib >> 1) & 1u) << 8 | ((nib >> 2) & 1u) << 16 |
                           ((nib >> 3) & 1u) << 24;
            }
            d[h] = make_uint4(parts[0], parts[1], parts[2], parts[3]);
        }
    }
}

__global__ void k_normalize(uint4 *__restrict__ p, uint64_t n_vec) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n_vec;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint4 w = p[v];
        uint32_t *parts = reinterpret_cast<uint32_t *>(&w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t x = parts[q];
            // per byte: 1 if non-zero
            x = (x | (x >> 4)) & 0x0f0f0f0fu;
            x = (x | (x >> 2)) & 0x03030303u;
            x = (x | (x >> 1)) & 0x01010101u;
            parts[q] = x;
        }
        p[v] = w;
    }
}

// ---------------------------------------------------------------------------------
// Baseline step kernel.
// ---------------------------------------------------------------------------------
template <bool kBitPacked>
struct SiteReader {
    const uint8_t *lat8;
    const uint32_t *latp;
    int L;
    __device__ __forceinline__ int operator()(int i, int j) const {
        i = wrap_near(i, L);
        j = wrap_near(j, L);
        if (kBitPacked) {
            return static_cast<int>((latp[static_cast<size_t>(i) * (L >> 5) + (j >> 5)] >> (j & 31)) &
                                    1u);
        } else {
            return lat8[static_cast<size_t>(i) * L + j];
        }
    }
};

// Sum of the cooperator counts of the five groups containing z = (i, j).
template <class Reader>
__device__ __forceinline__ int group_count_sum(const Reader &s, int i, int j) {
    const int near = s(i - 1, j) + s(i + 1, j) + s(i, j - 1) + s(i, j + 1);
    const int diag = s(i - 1, j - 1) + s(i - 1, j + 1) + s(i + 1, j - 1) + s(i + 1, j + 1);
    const int far = s(i - 2, j) + s(i + 2, j) + s(i, j - 2) + s(i, j + 2);
    return 5 * s(i, j) + 2 * (near + diag) + far;
}

// Number of cooperating nearest neighbours of z = (i, j) (the pairwise game, Section VI).
template <class Reader>
__device__ __forceinline__ int neighbour_count(const Reader &s, int i, int j) {
    return s(i - 1, j) + s(i + 1, j) + s(i, j - 1) + s(i, j + 1);
}

template <bool kBitPacked, int GAME>
__global__ void __launch_bounds__(256)
    k_step_simple(uint8_t *lat8, uint32_t *latp, int L, uint64_t seed, uint64_t k,
                  const uint32_t *__restrict__ table) {
    const int n4 = L >> 2;
    const int groups_per_row = (n4 + 7) >> 3;
    const long long tid = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (tid >= static_cast<long long>(n4) * groups_per_row) return;
    const int a = static_cast<int>(tid / groups_per_row);
    const int q = static_cast<int>(tid - static_cast<long long>(a) * groups_per_row);
    const int b0 = 8 * q;
    const int nb = min(8, n4 - b0);
    const int o = draw_offset(seed, k);
    const int oi = o >> 2, oj = o & 3;
    const int i = 4 * a + oi;
    const uint32_t dword = draw_dir_word(seed, k, a, b0);
    const SiteReader<kBitPacked> s{lat8, latp, L};

    uint4 u_lo = make_uint4(0, 0, 0, 0), u_hi = make_uint4(0, 0, 0, 0);
    bool have_lo = false, have_hi = false;
    uint32_t flips = 0;  // bit m: site b0 + m adopts
    for (int m = 0; m < nb; ++m) {
        const int b = b0 + m;
        const int j = 4 * b + oj;
        const int d = static_cast<int>((dword >> (2 * (b & 15))) & 3u);
        const int yi = i + (d == 2 ? 1 : (d == 3 ? -1 : 0));
        const int yj = j + (d == 0 ? 1 : (d == 1 ? -1 : 0));
        const int sx = s(i, j), sy = s(yi, yj);
        if (sx == sy) continue;
        uint32_t t;
        if constexpr (GAME == kPairGame) {
            const int nx = neighbour_count(s, i, j), ny = neighbour_count(s, yi, yj);
            t = __ldg(&table[(sx * kNRange + nx) * kNRange + ny]);
        } else {
            const int Sx = group_count_sum(s, i, j), Sy = group_count_sum(s, yi, yj);
            t = __ldg(&table[(sx * kSRange + Sx) * kSRange + Sy]);
        }
        uint32_t u;
        if (m < 4) {
            if (!have_lo) { u_lo = draw_u4(seed, k, a, (b0 >> 2)); have_lo = true; }
            u = word_of(u_lo, b & 3);
        } else {
            if (!have_hi) { u_hi = draw_u4(seed, k, a, (b0 >> 2) + 1); have_hi = true; }
            u = word_of(u_hi, b & 3);
        }
        if (u < t) flips |= 1u << m;
    }
    if (!flips) return;
    if (kBitPacked) {
        // the eight sites share word q of row i (column 4 b0 = 32 q); this thread is the
        // only writer of that word in this step
        uint32_t mask = 0;
#pragma unroll
        for (int m = 0; m < 8; ++m)
            if (flips & (1u << m)) mask |= 1u << (4 * m + oj);
        uint32_t *w = &latp[static_cast<size_t>(i) * (L >> 5) + q];
        *w ^= mask;
    } else {
        for (int m = 0; m < nb; ++m)
            if (flips & (1u << m)) {
                uint8_t *p = &lat8[static_cast<size_t>(i) * L + 4 * (b0 + m) + oj];
                *p ^= 1u;
            }
    }
}

int grid_for(uint64_t work, int block) {
    uint64_t g = (work + block - 1) / block;
    if (g > (1u << 20)) g = 1u << 20;
    if (g < 1) g = 1;
    return static_cast<int>(g);
}

}  // namespace

cudaError_t launch_init(int layout, void *lat, int L, uint64_t seed, uint64_t thr,
                        cudaStream_t s) {
    const uint64_t n = static_cast<uint64_t>(L) * L;
    if (layout == kU8) {
        k_init_u8<<<grid_for(n / 4, 256), 256, 0, s>>>(static_cast<uint8_t *>(lat), n / 4, seed, thr);
    } else {
        k_init_packed<<<grid_for(n / 32, 256), 256, 0, s>>>(static_cast<uint32_t *>(lat), n / 32,
                                                             seed, thr);
    }
    return cudaGetLastError();
}

cudaError_t launch_step_simple(int layout, int game, void *lat, int L, uint64_t seed, uint64_t k,
                               const uint32_t *table, cudaStream_t s) {
    const int n4 = L >> 2;
    const uint64_t threads = static_cast<uint64_t>(n4) * ((n4 + 7) >> 3);
    const int block = 256;
    const unsigned grid = static_cast<unsigned>((threads + block - 1) / block);
    uint8_t *l8 = layout == kU8 ? static_cast<uint8_t *>(lat) : nullptr;
    uint32_t *lp = layout == kU8 ? nullptr : static_cast<uint32_t *>(lat);
    if (game == kPairGame) {
        if (layout == kU8) k_step_simple<false, kPairGame><<<grid, block, 0, s>>>(l8, lp, L, seed, k, table);
        else k_step_simple<true, kPairGame><<<grid, block, 0, s>>>(l8, lp, L, seed, k, table);
    } else {
        if (layout == kU8) k_step_simple<false, kGroupGame><<<grid, block, 0, s>>>(l8, lp, L, seed, k, table);
        else k_step_simple<true, kGroupGame><<<grid, block, 0, s>>>(l8, lp, L, seed, k, table);
    }
    return cudaGetLastError();
}

cudaError_t launch_popcount(const void *buf, size_t bytes, unsigned long long *out,
                            cudaStream_t s) {
    const uint64_t n_vec = bytes / 16;
    k_popcount<<<grid_for(n_vec, 256) > 1216 ? 1216 : grid_for(n_vec, 256), 256, 0, s>>>(
        static_cast<const uint4 *>(buf), n_vec, out);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t *src, uint32_t *dst, int L, cudaStream_t s) {
    const uint64_t n_words = static_cast<uint64_t>(L) * L / 32;
    k_pack<<<grid_for(n_words, 256), 256, 0, s>>>(src, dst, n_words);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const uint32_t *src, uint8_t *dst, int L, cudaStream_t s) {
    const uint64_t n_words = static_cast<uint64_t>(L) * L / 32;
    k_unpack<<<grid_for(n_words, 256), 256, 0, s>>>(src, dst, n_words);
    return cudaGetLastError();
}

cudaError_t launch_normalize(uint8_t *buf, size_t n, cudaStream_t s) {
    const uint64_t n_vec = n / 16;
    k_normalize<<<grid_for(n_vec, 256), 256, 0, s>>>(reinterpret_cast<uint4 *>(buf), n_vec);
    return cudaGetLastError();
}

}  // namespace pgg
