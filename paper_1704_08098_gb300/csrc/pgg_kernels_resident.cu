// pgg_kernels_resident.cu -- a whole bit-packed lattice resident in shared memory across
// many MCS: one cooperative launch, each CTA owning a band of rows.
//
// CTA b keeps rows [r0, r1) of the lattice plus 3 halo rows above and below in shared memory
// for the whole call. A sublattice step writes only rows i = oi (mod 4), at least 4 apart, and
// an update reads rows i-3 .. i+3 (Section IV, Fig. 3), so within a step no CTA needs data a
// neighbour writes in that step; between steps each CTA publishes its 3 top and 3 bottom band
// rows to a double-buffered mailbox in global memory, bumps its step counter, and before the
// edge rows of the next step waits for both neighbours' counters and their rows in its halo.
// All CTAs are co-resident (cooperative launch). Every wait is bounded: after `spin_limit`
// polls the CTA sets the status word and stops; its neighbours then time out in turn.
//
// The exchange runs beside the computation: one extra warp per CTA polls the neighbours'
// counters, fetches their edge rows into the halo with TMA bulk copies (cp.async.bulk,
// completion on an mbarrier) and, after each step, bulk-stores the band's own edge rows and
// releases its counter, while the 16 compute warps update the interior rows; the compute
// warps wait on the mbarrier only before the edge rows.
//
// The pairwise game (Section VI) runs the same way with its radius-2 update (its halo rows
// beyond the second are exchanged but never read).
//
// Per step the work is the direct kernel's: tasks of one sublattice row and 1-4 words, the shared
// update core of pgg_unit.cuh, in place in shared memory. A step first updates the band's
// interior sublattice rows, whose reads stay inside the band, and only then waits for the
// neighbours and refreshes the halo for the at most two edge rows: the wait overlaps work (the
// edge rows go to the threads the interior leaves one task short). The count after each MCS is
// the sum of the bands' population counts. The band is staged with 4-byte cp.async copies and
// written back once per launch; a uint8 lattice is packed as its band is staged (two 16-byte
// loads per word) and unpacked as it is written back, so it needs no conversion launches.
#include <cuda_runtime.h>

#include "pgg_device.cuh"
#include "pgg_internal.h"
#include "pgg_unit.cuh"

namespace pgg {
namespace {

constexpr int kComputeThreads = 512;                 // warps that update the band
constexpr int kResThreads = kComputeThreads + 32;     // plus one warp that exchanges halos
constexpr int kResMaxUPT = 4;  // words per task at most (a task stays inside one 8-word direction call)

struct ResidentParams {
    uint32_t *lat;            // bit-packed global lattice (read at the start, written at the end)
    uint8_t *lat8;            // or, when not null, a uint8 lattice (lat unused)
    int L, Lw, n_bands;
    uint64_t seed, k0;
    int n_mcs;
    const uint32_t *table;
    uint32_t *mailbox;        // [band][parity][top/bottom][3 rows][Lw]
    unsigned int *ctr;        // [band] ctr_base + completed steps of this launch
    unsigned int ctr_base;    // above every value an earlier launch left in ctr
    unsigned long long *counts;  // [n_mcs], zeroed before the launch
    int *status;              // | 1 a wait timed out, | 2 misaligned buffers, | 4 an index check failed (checked build),
                              // | 8 a CTA stopped with a halo load possibly still in flight
    unsigned int spin_limit;
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

// Word w of a band row lives at (w ^ ((w >> 5) & 7)): the 32 lanes of a warp, which start
// tasks u = 1, 2 or 4 words apart (words u c, c = 0..31), then hit 32 different banks (for
// u = 4: bank 4 (c mod 8) + c / 8; for u = 2: 2c, or 2c - 31 for c >= 16).
__device__ __forceinline__ int swz(int w) { return w ^ ((w >> 5) & 7); }

__device__ __forceinline__ unsigned int load_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Sublattice rows of the band (global rows r in [r0, r0 + nb) with r = oi (mod 4)), split
// into the interior ones, whose reads (rows r-R .. r+R, R the game's read radius) stay inside
// the band, and the at most two edge ones that read halo rows.
struct BandRows {
    int first, n_srows, in_lo, in_hi;  // interior = sublattice rows in_lo .. in_hi - 1
};

template <int GAME>
__device__ __forceinline__ BandRows band_rows(int r0, int nb, int oi) {
    constexpr int R = kReadRadius<GAME>;
    BandRows b;
    b.first = r0 + ((oi - r0) & 3);
    b.n_srows = b.first < r0 + nb ? (r0 + nb - b.first + 3) >> 2 : 0;
    if (b.n_srows == 0) {
        b.in_lo = b.in_hi = 0;
        return b;
    }
    const int last = b.first + 4 * (b.n_srows - 1);
    b.in_lo = b.first - R < r0 ? 1 : 0;
    b.in_hi = last + R >= r0 + nb ? b.n_srows - 1 : b.n_srows;
    if (b.in_hi < b.in_lo) b.in_hi = b.in_lo;  // one sublattice row that is an edge row at both ends
    return b;
}

// Words per task of the interior phase: 4 when that still gives every thread a task, else
// fewer, so that small phases spread over all warps instead of a few long tasks.
__device__ __forceinline__ int interior_task_words(int words) {
    return words >= kResMaxUPT * kComputeThreads ? kResMaxUPT : (words >= 2 * kComputeThreads ? 2 : 1);
}

// Update the interior sublattice rows of the band (edge = false) or its edge rows (edge = true:
// row 0 when in_lo = 1, row n_srows - 1 when in_hi < n_srows; never the same row twice, since
// in_hi >= in_lo). Rows of one sublattice step are 4 apart and an update reads 3 rows either
// side, so the two calls touch disjoint sites and need no barrier between them.
//
// The interior tasks go to threads 0, 1, ... in turn, so when their number n_int is not a
// multiple of the thread count, threads f = n_int mod T and up have one task fewer. The edge
// tasks are dealt to those threads first (task e to thread f + e, wrapping), with as few words
// per task as still fit them: the edge rows then fill the gap of the last interior round instead
// of forming a round of their own.
template <int OJ, int GAME>
__device__ __forceinline__ void resident_step(uint32_t *s_rows, const uint32_t *__restrict__ s_table,
                                              const PhiloxKeys &rk, int Lw, int r0, int nb, const BandRows &br,
                                              bool edge, uint64_t k, int *status) {
    const long long n_local = static_cast<long long>(nb + 6) * Lw;  // words of band + halo
    // edge: selected row q is 0 or n_srows - 1 (edge_top: whether row 0 is one of them)
    const bool edge_top = br.in_lo != 0, edge_bot = br.in_hi < br.n_srows;
    const int n_rows_sel = edge ? static_cast<int>(edge_top) + static_cast<int>(edge_bot) : br.in_hi - br.in_lo;
    const int words = n_rows_sel * Lw;
    int upt, shift = 0;
    if (edge) {
        const int int_words = (br.in_hi - br.in_lo) * Lw;
        const int f = (int_words / interior_task_words(int_words)) % kComputeThreads;
        const int free_threads = f ? kComputeThreads - f : kComputeThreads;
        upt = words <= free_threads ? 1 : (words <= 2 * free_threads ? 2 : kResMaxUPT);
        shift = f;
    } else {
        upt = interior_task_words(words);
    }
    const int runs = Lw / upt;
    const int n_tasks = n_rows_sel * runs;
    const uint32_t kl = static_cast<uint32_t>(k), kh = static_cast<uint32_t>(k >> 32) | kTagDir;
    int t0 = static_cast<int>(threadIdx.x) - shift;
    if (t0 < 0) t0 += kComputeThreads;
    for (int t = t0; t < n_tasks; t += kComputeThreads) {
        const int q_sel = t / runs;
        const int sr = edge ? ((q_sel == 0 && edge_top) ? 0 : br.n_srows - 1) : br.in_lo + q_sel;
        const int c = t - q_sel * runs;
        const int i = br.first + 4 * sr;         // global row
        const int lr = i - r0 + 3;               // local row (3 halo rows above the band)
        const uint32_t *row0 = s_rows + (lr - 3) * Lw;
        const int w0 = upt * c;
        const int wprev = w0 == 0 ? Lw - 1 : w0 - 1;
        uint32_t wl[7], wc[7], wr[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const long long base = static_cast<long long>(lr - 3 + q) * Lw;
            wl[q] = reads_row<GAME>(q) && index_ok(base + swz(wprev), n_local, status) ? row0[q * Lw + swz(wprev)] : 0u;
            wc[q] = reads_row<GAME>(q) && index_ok(base + swz(w0), n_local, status) ? row0[q * Lw + swz(w0)] : 0u;
        }
        const uint4 dcall = philox_rk(make_uint4(static_cast<uint32_t>(w0 >> 3), static_cast<uint32_t>(i >> 2), kl, kh), rk);
        UnitCtx u;
        u.k = k;
        u.a = static_cast<uint32_t>(i >> 2);
        u.msk = kNib;
#pragma unroll 1
        for (int w = w0; w < w0 + upt; ++w) {
            const int wn = w + 1 == Lw ? 0 : w + 1;
#pragma unroll
            for (int q = 0; q < 7; ++q)
                wr[q] = reads_row<GAME>(q) && index_ok(static_cast<long long>(lr - 3 + q) * Lw + swz(wn), n_local, status)
                            ? row0[q * Lw + swz(wn)]
                            : 0u;
            u.gw = w;
            u.d16 = (word_of(dcall, (w >> 1) & 3) >> (16 * (w & 1))) & 0xFFFFu;
            uint32_t sx;
            const uint32_t flips = game_flips<OJ, GAME>(wl, wc, wr, u, rk, s_table, sx);
            // writes stay in the band's own rows (local rows 3 .. nb + 2)
            if (flips && index_ok(lr - 3, nb, status)) s_rows[lr * Lw + swz(w)] = wc[3] ^ (flips << OJ);
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                wl[q] = wc[q];
                wc[q] = wr[q];
            }
        }
    }
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
__device__ __forceinline__ void copy_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Barrier of the compute warps only (the communication warp does not take part).
__device__ __forceinline__ void compute_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(kComputeThreads) : "memory"); }

// try_wait calls a compute warp makes on the halo mbarrier before it gives up (each call may
// suspend the thread for a short time; a bulk copy from L2 lands within microseconds).
constexpr unsigned int kMbarTries = 1u << 26;

template <int GAME>
__global__ void __launch_bounds__(kResThreads, 1) k_resident(const __grid_constant__ ResidentParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *s_table = smem;
    uint32_t *s_rows = smem + kTableEntries;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ volatile int s_abort;
    __shared__ unsigned long long s_warp[kComputeThreads / 32];
    const int tid = threadIdx.x;
    const bool comm = tid >= kComputeThreads;  // the last warp exchanges halos, the others compute
    const int b = blockIdx.x, nbnd = p.n_bands;
    const int L = p.L, Lw = p.Lw;
    const int r0 = band_start(b, L, nbnd), nb = band_start(b + 1, L, nbnd) - r0;
    const int up = (b + nbnd - 1) % nbnd, down = (b + 1) % nbnd;
    const size_t edge = static_cast<size_t>(3) * Lw;                  // words of 3 rows
    const uint32_t edge_bytes = static_cast<uint32_t>(edge * sizeof(uint32_t));
    const PhiloxKeys rk = p.rk;
    // bulk copies need 16-byte aligned rows (the same answer in every CTA: all stop together)
    if ((smem_u32(s_rows) & 15u) != 0u || (reinterpret_cast<uintptr_t>(p.mailbox) & 15u) != 0u ||
        (reinterpret_cast<uintptr_t>(p.lat8) & 15u) != 0u) {
        if (tid == 0) atomicOr(p.status, 2);
        return;
    }
    for (int t = tid; t < kTableEntries; t += kResThreads) copy_async4(&s_table[t], &p.table[t]);
    if (tid == 0) {
        s_abort = 0;
        mbar_init(&s_mbar, 1);
    }
    // stage the table and band + halo (rows r0 - 3 .. r0 + nb + 2, periodic) with 4-byte
    // asynchronous copies (cp.async: many loads in flight per thread, each word to its place);
    // thread t copies column t mod Lw of every (T / Lw)-th row, so a copy costs a few adds
    const int rows_per_pass = kResThreads / Lw;   // >= 1: a resident row has at most 448 words
    const int col = tid % Lw, row_first = tid / Lw;
    const int scol = swz(col);
    if (row_first < rows_per_pass) {
        int g = wrap_small(r0 - 3 + row_first, L);
        if (p.lat8) {
            // uint8 lattice: the word's 32 bytes in two 16-byte loads (rows start 256-byte aligned)
#pragma unroll 4
            for (int lr = row_first; lr < nb + 6; lr += rows_per_pass) {
                const size_t off = static_cast<size_t>(g) * L + 32 * static_cast<size_t>(col);
                if (index_ok(static_cast<long long>(off) + 31, static_cast<long long>(L) * L, p.status)) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(p.lat8 + off);
                    s_rows[lr * Lw + scol] = pack_bytes32(src[0], src[1]);
                }
                g += rows_per_pass;
                if (g >= L) g -= L;
            }
        } else {
            for (int lr = row_first; lr < nb + 6; lr += rows_per_pass) {
                if (index_ok(static_cast<long long>(g) * Lw + col, static_cast<long long>(L) * Lw, p.status))
                    copy_async4(&s_rows[lr * Lw + scol], &p.lat[static_cast<size_t>(g) * Lw + col]);
                g += rows_per_pass;
                if (g >= L) g -= L;
            }
        }
    }
    copy_async_wait_all();
    fence_async_shared();  // the staged halo rows are later overwritten by bulk loads
    __syncthreads();
    uint4 ocall = make_uint4(0, 0, 0, 0);
    uint64_t ocall_idx = ~0ull;
    const int total = 16 * p.n_mcs;
    bool load_pending = false;  // communication lane: a halo load not yet seen complete
    for (int j = 0; j < total; ++j) {
        const uint64_t k = p.k0 + static_cast<uint64_t>(j);
        if (comm) {
            // fetch the neighbours' rows after step j - 1 into the halo, asynchronously
            if (tid == kComputeThreads && j > 0) {
                unsigned int it = 0;
                const unsigned int want = p.ctr_base + static_cast<unsigned int>(j);
                while ((load_acquire(&p.ctr[up]) < want || load_acquire(&p.ctr[down]) < want) && it < p.spin_limit) {
                    __nanosleep(32);
                    ++it;
                }
                if (it >= p.spin_limit) {
                    atomicOr(p.status, 1);
                    s_abort = 1;
                } else {
                    const int par = (j - 1) & 1;
                    const uint32_t *from_up = p.mailbox + ((static_cast<size_t>(up) * 2 + par) * 2 + 1) * edge;
                    const uint32_t *from_down = p.mailbox + ((static_cast<size_t>(down) * 2 + par) * 2 + 0) * edge;
                    fence_async_global();  // the acquired rows, for the async proxy's reads
                    mbar_expect_tx(&s_mbar, 2 * edge_bytes);
                    bulk_load(s_rows, from_up, edge_bytes, &s_mbar);
                    bulk_load(s_rows + static_cast<size_t>(nb + 3) * Lw, from_down, edge_bytes, &s_mbar);
                    load_pending = true;
                }
            }
            __syncwarp();
        } else {
            if ((k >> 5) != ocall_idx) {
                ocall_idx = k >> 5;
                ocall = philox_rk(make_uint4(static_cast<uint32_t>(ocall_idx), static_cast<uint32_t>(ocall_idx >> 32), 0u,
                                             kTagOffset), rk);
            }
            const int o = static_cast<int>((word_of(ocall, static_cast<int>((k >> 3) & 3)) >> (4 * (k & 7))) & 15u);
            const BandRows br = band_rows<GAME>(r0, nb, o >> 2);
            // interior rows read only the band's own rows: they run while the halo is in flight
            switch (o & 3) {
                case 0: resident_step<0, GAME>(s_rows, s_table, rk, Lw, r0, nb, br, false, k, p.status); break;
                case 1: resident_step<1, GAME>(s_rows, s_table, rk, Lw, r0, nb, br, false, k, p.status); break;
                case 2: resident_step<2, GAME>(s_rows, s_table, rk, Lw, r0, nb, br, false, k, p.status); break;
                default: resident_step<3, GAME>(s_rows, s_table, rk, Lw, r0, nb, br, false, k, p.status); break;
            }
            bool ready = true;
            if (j > 0) {
                unsigned int it = 0;
                while (!mbar_try_wait(&s_mbar, static_cast<uint32_t>((j - 1) & 1))) {
                    if (s_abort || ++it >= kMbarTries) {
                        ready = false;
                        break;
                    }
                }
            }
            if (ready) {
                // the at most two edge rows, which read the halo
                switch (o & 3) {
                    case 0: resident_step<0, GAME>(s_rows, s_table, rk, Lw, r0, nb, br, true, k, p.status); break;
                    case 1: resident_step<1, GAME>(s_rows, s_table, rk, Lw, r0, nb, br, true, k, p.status); break;
                    case 2: resident_step<2, GAME>(s_rows, s_table, rk, Lw, r0, nb, br, true, k, p.status); break;
                    default: resident_step<3, GAME>(s_rows, s_table, rk, Lw, r0, nb, br, true, k, p.status); break;
                }
            } else {
                s_abort = 1;
            }
            fence_async_shared();  // this thread's lattice writes, for the bulk store below
        }
        __syncthreads();
        if (s_abort) {
            // a wait ran out: make sure no bulk copy still targets this CTA's shared memory,
            // then stop; the lattice in global memory is left as it was
            if (tid == kComputeThreads && load_pending) {
                unsigned int it = 0;
                while (!mbar_try_wait(&s_mbar, static_cast<uint32_t>((j - 1) & 1)) && ++it < kMbarTries) {
                }
                // the halo load was never seen to land: the CTA leaves with a copy into its
                // shared memory possibly in flight, which the host must treat as fatal
                if (it >= kMbarTries) atomicOr(p.status, 8);
            }
            return;
        }
        load_pending = false;
        if (comm) {
            // publish the band's top and bottom 3 rows (as laid out in shared memory) for the
            // neighbours' next step; the compute warps meanwhile start step j + 1, which
            // writes neither
            if (tid == kComputeThreads) {
                uint32_t *to_top = p.mailbox + ((static_cast<size_t>(b) * 2 + (j & 1)) * 2 + 0) * edge;
                uint32_t *to_bot = p.mailbox + ((static_cast<size_t>(b) * 2 + (j & 1)) * 2 + 1) * edge;
                bulk_store(to_top, s_rows + static_cast<size_t>(3) * Lw, edge_bytes);
                bulk_store(to_bot, s_rows + static_cast<size_t>(nb) * Lw, edge_bytes);
                bulk_commit_and_wait();
                fence_async_global();
                __threadfence();
                store_release(&p.ctr[b], p.ctr_base + static_cast<unsigned int>(j + 1));
            }
            __syncwarp();
        } else if ((j & 15) == 15 && p.counts) {
            unsigned long long c = 0;
            for (int x = tid; x < nb * Lw; x += kComputeThreads) c += __popc(s_rows[3 * Lw + x]);
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) c += __shfl_down_sync(0xffffffffu, c, s);
            if ((tid & 31) == 0) s_warp[tid >> 5] = c;
            compute_barrier();
            if (tid == 0) {
                unsigned long long tot = 0;
                for (int w = 0; w < kComputeThreads / 32; ++w) tot += s_warp[w];
                atomicAdd(&p.counts[j >> 4], tot);
            }
        }
    }
    __syncthreads();  // the last bulk store has completed (its issuer waited) before the band is stored
    // store the band (the same column-per-thread walk)
    if (row_first < rows_per_pass) {
        if (p.lat8) {
            for (int lr = row_first; lr < nb; lr += rows_per_pass) {
                const size_t off = static_cast<size_t>(r0 + lr) * L + 32 * static_cast<size_t>(col);
                if (index_ok(static_cast<long long>(off) + 31, static_cast<long long>(L) * L, p.status)) {
                    const uint32_t w = s_rows[(lr + 3) * Lw + scol];
                    uint4 *dst = reinterpret_cast<uint4 *>(p.lat8 + off);
                    dst[0] = unpack_bits16(w & 0xFFFFu);
                    dst[1] = unpack_bits16(w >> 16);
                }
            }
        } else {
            for (int lr = row_first; lr < nb; lr += rows_per_pass) {
                if (index_ok(static_cast<long long>(r0 + lr) * Lw + col, static_cast<long long>(L) * Lw, p.status))
                    p.lat[static_cast<size_t>(r0 + lr) * Lw + col] = s_rows[(lr + 3) * Lw + scol];
            }
        }
    }
}

}  // namespace

// Bands for a lattice of side L: one per SM when every band keeps at least 4 rows and its
// rows fit the shared memory; 0 when the lattice cannot be resident. The kernel works on the
// bit-packed form; a uint8 lattice is packed for the call by the caller.
int resident_bands(int layout, int L, int sms, size_t smem_optin) {
    (void)layout;
    if (L < 256 || L % 256 != 0 || sms < 1) return 0;
    int n = sms;
    while (n > 1 && L / n < 4) --n;
    const int max_rows = (L + n - 1) / n;
    const size_t need = sizeof(uint32_t) * (kTableEntries + static_cast<size_t>(max_rows + 6) * (L / 32));
    return need <= smem_optin ? n : 0;
}

size_t resident_mailbox_words(int L, int n_bands) { return static_cast<size_t>(n_bands) * 2 * 2 * 3 * (L / 32); }

cudaError_t launch_resident(const ResidentArgs &a, cudaStream_t s) {
    if (a.n_bands < 1 || a.L % 256 != 0) return cudaErrorInvalidValue;
    ResidentParams p;
    p.lat = a.lat;
    p.lat8 = a.lat8;
    p.L = a.L;
    p.Lw = a.L / 32;
    p.n_bands = a.n_bands;
    p.seed = a.seed;
    p.k0 = a.k0;
    p.n_mcs = a.n_mcs;
    p.table = a.table;
    p.mailbox = a.mailbox;
    p.ctr = a.ctr;
    p.ctr_base = a.ctr_base;
    p.counts = a.counts;
    p.status = a.status;
    p.spin_limit = a.spin_limit;
    p.rk = philox_round_keys(a.seed);
    const int max_rows = (a.L + a.n_bands - 1) / a.n_bands;
    const size_t smem = sizeof(uint32_t) * (kTableEntries + static_cast<size_t>(max_rows + 6) * p.Lw);
    const void *kernel = a.game == kPairGame ? reinterpret_cast<const void *>(k_resident<kPairGame>)
                                             : reinterpret_cast<const void *>(k_resident<kGroupGame>);
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
