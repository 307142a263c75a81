// pgg_batch.cu -- many independent replicas (different L, r, K, seed) advanced in one
// persistent launch, each replica's bit-packed lattice resident in shared memory for the
// whole run.
//
// A replica of side L <= 1024 needs L^2 / 8 <= 128 KB, so it fits in one SM's shared memory.
// One 1024-thread CTA per SM pulls jobs from an atomic queue (largest first). A job is a
// group of replicas of one size packed into the CTA's 32 warps and 128 KB: a "team" of warps
// advances each replica (1, 1, 2, 8, 32 warps for L = 64, 128, 256, 512, 1024 by default,
// i.e. at most 8 word units per thread per sublattice step), synchronising with a named
// barrier between sublattice steps. The team loads the lattice once, runs all n_mcs MCS
// (16 sublattice steps each, the same update rule and random stream as the single-lattice
// kernels), writes the cooperator count after every MCS, and stores the lattice back. A replica
// whose count reaches 0 or L^2 is in an absorbing state (all D or all C: every neighbour holds the
// site's own strategy, so no update can change it): its team writes that count for the remaining
// MCS and stops, which gives the same lattice, step counter and counts as running them.
//
// Shared-memory layout of a replica: row-major words with a per-row rotation,
// word (row, w) at row * Lw + (w + row) mod Lw, so that the threads of a warp, which work
// on consecutive rows, hit distinct banks (Lw is even, Lw + 1 is odd).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pgg.h"
#include "pgg_device.cuh"
#include "pgg_internal.h"
#include "pgg_unit.cuh"

namespace pgg {
namespace {

constexpr int kBatchMaxWarps = 32;  // largest CTA: 1024 threads
constexpr int kBatchMaxL = 1024;
constexpr size_t kBatchSmemBytes = size_t(kBatchMaxL) * kBatchMaxL / 8;  // 128 KB
constexpr int kSizeClasses = 5;                                         // L = 64 .. 1024

struct ReplicaDesc {
    uint32_t *lat;          // bit-packed lattice in global memory (L rows of L/32 words)
    const uint32_t *table;  // 2*26*26 thresholds of this replica's (r, K)
    uint64_t seed;
    uint64_t step;          // sublattice step counter, advanced by the kernel
    int L;
    int pad;
    PhiloxKeys rk;
};

// Initial condition of every replica in one launch: blockIdx.y strides over the replicas,
// the x blocks over the words of one replica (smaller replicas leave blocks idle).
__global__ void k_batch_init(const ReplicaDesc *__restrict__ desc, int n, uint64_t thr) {
    for (int i = blockIdx.y; i < n; i += gridDim.y) {
        const ReplicaDesc d = desc[i];
        const uint64_t n_words = static_cast<uint64_t>(d.L) * d.L / 32;
        for (uint64_t wi = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; wi < n_words;
             wi += static_cast<uint64_t>(gridDim.x) * blockDim.x)
            d.lat[wi] = init_packed_word(wi, d.seed, thr);
    }
}

struct Job {
    int first;       // index into members[]
    int n_teams;     // replicas in the job
    int team_warps;  // warps per replica
    int L;
};

struct BatchParams {
    ReplicaDesc *replicas;
    const int *members;      // replica ids, grouped by job
    const Job *jobs;
    int n_jobs;
    int n_mcs;
    unsigned int *job_counter;  // zeroed before each launch
    uint32_t *counts;           // [replica][n_mcs] cooperator counts (nullable)
};

template <int CTA_WARPS>
__device__ __forceinline__ void team_sync(int team, int team_warps) {
    if (team_warps == 1) {
        __syncwarp();
    } else if (team_warps == CTA_WARPS) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(team_warps * 32) : "memory");
    }
}

// One sublattice step of a shared-memory-resident replica, column offset OJ.
template <int OJ>
__device__ __forceinline__ long long batch_step(uint32_t *s_lat, const uint32_t *__restrict__ table, const PhiloxKeys &rk,
                                                int L, int Lw, uint64_t k, int oi, int tid, int nthr) {
    const int runs = (Lw + 7) >> 3;          // call-aligned runs of 8 words per row (power of 2)
    const int runs_log2 = 31 - __clz(runs);
    const int n_tasks = (L >> 2) * runs;
    const int wmask = Lw - 1;                // Lw is a power of two
    const uint32_t kl = static_cast<uint32_t>(k), kh = static_cast<uint32_t>(k >> 32) | kTagDir;
    long long delta = 0;
    for (int t = tid; t < n_tasks; t += nthr) {
        const int a = t >> runs_log2;
        const int c = t & (runs - 1);
        const int i = 4 * a + oi;
        int rowbase[7], rot[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const int row = wrap_small(i - 3 + q, L);
            rowbase[q] = row * Lw;
            rot[q] = row & wmask;
        }
        const int w0 = 8 * c;
        const int w1 = min(w0 + 8, Lw);
        auto at = [&](int q, int w) -> uint32_t { return s_lat[rowbase[q] + ((w + rot[q]) & wmask)]; };
        const int wprev = w0 == 0 ? Lw - 1 : w0 - 1;
        uint32_t wl[7], wc[7], wr[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            wl[q] = at(q, wprev);
            wc[q] = at(q, w0);
        }
        const uint4 dcall = philox_rk(make_uint4(static_cast<uint32_t>(c), static_cast<uint32_t>(a), kl, kh), rk);
        UnitCtx u;
        u.k = k;
        u.a = static_cast<uint32_t>(a);
        u.msk = kNib;
#pragma unroll 1
        for (int w = w0; w < w1; ++w) {
            const int wn = w + 1 == Lw ? 0 : w + 1;
#pragma unroll
            for (int q = 0; q < 7; ++q) wr[q] = at(q, wn);
            u.gw = w;
            u.d16 = (word_of(dcall, (w >> 1) & 3) >> (16 * (w & 1))) & 0xFFFFu;
            uint32_t sx;
            const uint32_t flips = unit_flips<OJ>(wl, wc, wr, u, rk, table, sx);
            if (flips) {
                s_lat[rowbase[3] + ((w + rot[3]) & wmask)] = wc[3] ^ (flips << OJ);
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

template <int CTA_THREADS>
__global__ void __launch_bounds__(CTA_THREADS, 1) k_batch(const __grid_constant__ BatchParams p) {
    constexpr int kWarps = CTA_THREADS / 32;
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_job;
    __shared__ unsigned long long s_count[2][kWarps];  // per team, by MCS parity
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_job = static_cast<int>(atomicAdd(p.job_counter, 1u));
        __syncthreads();
        const int job = s_job;
        if (job >= p.n_jobs) break;
        const Job J = p.jobs[job];
        const int team = warp / J.team_warps;
        if (team < J.n_teams) {
            const int rid = p.members[J.first + team];
            const ReplicaDesc &d = p.replicas[rid];
            const int L = J.L, Lw = L >> 5, words = L * Lw;
            const int tid = threadIdx.x - team * J.team_warps * 32, nthr = J.team_warps * 32;
            uint32_t *s_lat = smem + team * words;
            const PhiloxKeys rk = d.rk;
            const uint64_t step0 = d.step;
            const uint32_t *table = d.table;
            uint32_t *glat = d.lat;
            const int lw_log2 = 31 - __clz(Lw);
            // stage the lattice (rotated rows)
            for (int x = tid; x < words; x += nthr) {
                const int row = x >> lw_log2, w = x & (Lw - 1);
                s_lat[(row << lw_log2) + ((w + row) & (Lw - 1))] = glat[x];
            }
            if (tid == 0) {
                s_count[0][team] = 0;
                s_count[1][team] = 0;
            }
            team_sync<kWarps>(team, J.team_warps);
            uint64_t k = step0;
            uint4 ocall = make_uint4(0, 0, 0, 0);
            uint64_t ocall_idx = ~0ull;
            for (int m = 0; m < p.n_mcs; ++m) {
                for (int s = 0; s < 16; ++s, ++k) {
                    if ((k >> 5) != ocall_idx) {
                        ocall_idx = k >> 5;
                        ocall = philox_rk(make_uint4(static_cast<uint32_t>(ocall_idx), static_cast<uint32_t>(ocall_idx >> 32),
                                                     0u, kTagOffset), rk);
                    }
                    const int o = static_cast<int>((word_of(ocall, static_cast<int>((k >> 3) & 3)) >> (4 * (k & 7))) & 15u);
                    switch (o & 3) {
                        case 0: batch_step<0>(s_lat, table, rk, L, Lw, k, o >> 2, tid, nthr); break;
                        case 1: batch_step<1>(s_lat, table, rk, L, Lw, k, o >> 2, tid, nthr); break;
                        case 2: batch_step<2>(s_lat, table, rk, L, Lw, k, o >> 2, tid, nthr); break;
                        default: batch_step<3>(s_lat, table, rk, L, Lw, k, o >> 2, tid, nthr); break;
                    }
                    team_sync<kWarps>(team, J.team_warps);
                }
                if (p.counts) {
                    unsigned long long c = 0;
                    for (int x = tid; x < words; x += nthr) c += __popc(s_lat[x]);
#pragma unroll
                    for (int sh = 16; sh > 0; sh >>= 1) c += __shfl_down_sync(0xffffffffu, c, sh);
                    if (lane == 0) atomicAdd(&s_count[m & 1][team], c);
                    team_sync<kWarps>(team, J.team_warps);
                    const unsigned long long cnt = s_count[m & 1][team];
                    // the other slot was last read after the previous MCS, 16 team barriers ago
                    if (tid == 0) s_count[(m + 1) & 1][team] = 0;
                    uint32_t *row = p.counts + static_cast<size_t>(rid) * p.n_mcs;
                    if (tid == 0) row[m] = static_cast<uint32_t>(cnt);
                    if (cnt == 0 || cnt == static_cast<unsigned long long>(words) * 32) {
                        // absorbing: the remaining MCS leave the lattice as it is
                        for (int m2 = m + 1 + tid; m2 < p.n_mcs; m2 += nthr) row[m2] = static_cast<uint32_t>(cnt);
                        break;
                    }
                }
            }
            // store the lattice back (undo the rotation)
            for (int x = tid; x < words; x += nthr) {
                const int row = x >> lw_log2, w = x & (Lw - 1);
                glat[x] = s_lat[(row << lw_log2) + ((w + row) & (Lw - 1))];
            }
            if (tid == 0) p.replicas[rid].step = step0 + 16ull * static_cast<uint64_t>(p.n_mcs);
        }
        __syncthreads();  // the job's shared memory is free again
    }
}

int size_class(int L) {
    switch (L) {
        case 64: return 0;
        case 128: return 1;
        case 256: return 2;
        case 512: return 3;
        case 1024: return 4;
        default: return -1;
    }
}

thread_local char g_batch_err[256];

}  // namespace
}  // namespace pgg

using pgg::Job;
using pgg::ReplicaDesc;

struct pgg_batch {
    int n = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<int> L;
    std::vector<double> r, K;
    std::vector<uint64_t> seeds;
    std::vector<ReplicaDesc> host_desc;
    ReplicaDesc *desc_d = nullptr;
    uint32_t *lat_pool = nullptr;   // all lattices, bit-packed, back to back
    uint32_t *table_pool = nullptr; // n tables
    int *members_d = nullptr;
    Job *jobs_d = nullptr;
    int n_jobs = 0;
    unsigned int *counter_d = nullptr;
    uint32_t *counts_d = nullptr;
    int64_t counts_cap = 0;
    // the autotuner's usual choice on GB300 (the 1024-thread CTA has 64 registers a thread and spills)
    int team_warps[pgg::kSizeClasses] = {1, 1, 2, 4, 16};
    int cta_threads = 512;
    // CUDA graph of one persistent launch (counter reset + kernel) for graph_n_mcs MCS
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_n_mcs = -1;
    bool graph_counts = false;
    bool use_graph = true;
    bool jobs_valid = false;
    int sms = 0;
};

namespace {

int bfail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return pgg::record_error(code, buf);
}

#define PGG_BCUDA(call)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return bfail(PGG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Pack replicas into jobs: replicas of one size, as many per job as fit the CTA's warps
// and 128 KB; jobs ordered by work per thread (largest first).
int build_jobs(pgg_batch *b) {
    std::vector<int> members;
    std::vector<Job> jobs;
    struct Cls { int L; std::vector<int> ids; };
    std::vector<Cls> cls;
    for (int c = pgg::kSizeClasses - 1; c >= 0; --c) {
        const int L = 64 << c;
        Cls k{L, {}};
        for (int i = 0; i < b->n; ++i)
            if (b->L[i] == L) k.ids.push_back(i);
        if (!k.ids.empty()) cls.push_back(k);
    }
    std::vector<std::pair<double, Job>> order;
    for (const auto &k : cls) {
        const int c = pgg::size_class(k.L);
        const int tw = b->team_warps[c];
        const size_t bytes = size_t(k.L) * k.L / 8;
        const int cta_warps = b->cta_threads / 32;
        int per_job = std::min<int>(cta_warps / tw, static_cast<int>(pgg::kBatchSmemBytes / bytes));
        if (tw > 1 && tw < cta_warps) per_job = std::min(per_job, 15);  // named barriers 1..15
        if (per_job < 1) per_job = 1;
        for (size_t s = 0; s < k.ids.size(); s += per_job) {
            Job j;
            j.first = static_cast<int>(members.size());
            j.n_teams = static_cast<int>(std::min<size_t>(per_job, k.ids.size() - s));
            j.team_warps = tw;
            j.L = k.L;
            for (int t = 0; t < j.n_teams; ++t) members.push_back(k.ids[s + t]);
            // work per thread of the job: sites / (16 threads-per-unit...) ~ L^2 / (team threads)
            const double work = double(k.L) * k.L / (tw * 32.0);
            order.push_back({work, j});
        }
    }
    std::stable_sort(order.begin(), order.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    for (const auto &o : order) jobs.push_back(o.second);
    if (b->members_d) cudaFree(b->members_d);
    if (b->jobs_d) cudaFree(b->jobs_d);
    b->members_d = nullptr;
    b->jobs_d = nullptr;
    PGG_BCUDA(cudaMalloc(&b->members_d, members.size() * sizeof(int)));
    PGG_BCUDA(cudaMalloc(&b->jobs_d, jobs.size() * sizeof(Job)));
    PGG_BCUDA(cudaMemcpyAsync(b->members_d, members.data(), members.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    PGG_BCUDA(cudaMemcpyAsync(b->jobs_d, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice, b->stream));
    PGG_BCUDA(cudaStreamSynchronize(b->stream));
    b->n_jobs = static_cast<int>(jobs.size());
    b->jobs_valid = true;
    b->graph_n_mcs = -1;
    return PGG_OK;
}

void drop_graph(pgg_batch *b) {
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
    b->graph_n_mcs = -1;
}

// Enqueue one persistent launch (counter reset + kernel) on stream s.
cudaError_t enqueue_launch(pgg_batch *b, int n_mcs, bool with_counts, cudaStream_t s) {
    pgg::BatchParams p;
    p.replicas = b->desc_d;
    p.members = b->members_d;
    p.jobs = b->jobs_d;
    p.n_jobs = b->n_jobs;
    p.n_mcs = n_mcs;
    p.job_counter = b->counter_d;
    p.counts = with_counts ? b->counts_d : nullptr;
    cudaError_t e = cudaMemsetAsync(b->counter_d, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int grid = std::min(b->sms > 0 ? b->sms : 1, b->n_jobs);
    if (b->cta_threads == 512)
        pgg::k_batch<512><<<grid, 512, pgg::kBatchSmemBytes, s>>>(p);
    else
        pgg::k_batch<1024><<<grid, 1024, pgg::kBatchSmemBytes, s>>>(p);
    return cudaGetLastError();
}

size_t lattice_words(int L) { return size_t(L) * L / 32; }

}  // namespace

extern "C" {

int pgg_batch_create(pgg_batch **out, int n, const int *L, const double *r, const double *K,
                     const uint64_t *seeds, void *cuda_stream) {
    pgg::clear_error();
    if (!out) return bfail(PGG_ERR_ARG, "pgg_batch_create: out is NULL");
    *out = nullptr;
    if (n < 1 || !L || !r || !K || !seeds) return bfail(PGG_ERR_ARG, "pgg_batch_create: need n >= 1 and all arrays");
    for (int i = 0; i < n; ++i) {
        if (pgg::size_class(L[i]) < 0)
            return bfail(PGG_ERR_ARG, "pgg_batch_create: replica %d has L = %d; batched replicas need L in {64, 128, 256, 512, 1024}", i, L[i]);
        if (!(r[i] > 0.0) || !std::isfinite(r[i]) || !(K[i] > 0.0) || !std::isfinite(K[i]))
            return bfail(PGG_ERR_ARG, "pgg_batch_create: replica %d needs r > 0 and K > 0", i);
    }
    pgg_batch *b = new (std::nothrow) pgg_batch();
    if (!b) return bfail(PGG_ERR_OOM, "pgg_batch_create: host allocation failed");
    b->n = n;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->L.assign(L, L + n);
    b->r.assign(r, r + n);
    b->K.assign(K, K + n);
    b->seeds.assign(seeds, seeds + n);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    size_t total_words = 0;
    for (int i = 0; i < n; ++i) total_words += lattice_words(L[i]);
    if (e == cudaSuccess) e = cudaMalloc(&b->lat_pool, total_words * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->table_pool, size_t(n) * pgg::kTableEntries * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->desc_d, size_t(n) * sizeof(ReplicaDesc));
    if (e == cudaSuccess) e = cudaMalloc(&b->counter_d, sizeof(unsigned int));
    if (e != cudaSuccess) {
        pgg_batch_destroy(b);
        return bfail(PGG_ERR_OOM, "pgg_batch_create: %s", cudaGetErrorString(e));
    }
    std::vector<uint32_t> tables(size_t(n) * pgg::kTableEntries);
    b->host_desc.resize(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        pgg::build_threshold_table(r[i], K[i], tables.data() + size_t(i) * pgg::kTableEntries);
        ReplicaDesc &d = b->host_desc[i];
        d.lat = b->lat_pool + off;
        d.table = b->table_pool + size_t(i) * pgg::kTableEntries;
        d.seed = seeds[i];
        d.step = 0;
        d.L = L[i];
        d.pad = 0;
        d.rk = pgg::philox_round_keys(seeds[i]);
        off += lattice_words(L[i]);
    }
    if ((e = cudaMemcpyAsync(b->table_pool, tables.data(), tables.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->desc_d, b->host_desc.data(), size_t(n) * sizeof(ReplicaDesc), cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->lat_pool, 0, total_words * sizeof(uint32_t), b->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(b->stream)) != cudaSuccess) {
        pgg_batch_destroy(b);
        return bfail(PGG_ERR_CUDA, "pgg_batch_create: %s", cudaGetErrorString(e));
    }
    e = cudaFuncSetAttribute(pgg::k_batch<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(pgg::kBatchSmemBytes));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pgg::k_batch<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(pgg::kBatchSmemBytes));
    if (e != cudaSuccess) {
        pgg_batch_destroy(b);
        return bfail(PGG_ERR_CUDA, "pgg_batch_create: shared memory attribute: %s", cudaGetErrorString(e));
    }
    *out = b;
    return PGG_OK;
}

int pgg_batch_seed(pgg_batch *b, double p) {
    pgg::clear_error();
    if (!b) return bfail(PGG_ERR_ARG, "pgg_batch_seed: NULL batch");
    if (!(p >= 0.0 && p <= 1.0)) return bfail(PGG_ERR_ARG, "pgg_batch_seed: p must be in [0, 1]");
    PGG_BCUDA(cudaSetDevice(b->device));
    const uint64_t thr = p >= 1.0 ? (1ull << 32) : static_cast<uint64_t>(p * 4294967296.0);
    int max_L = 0;
    for (int i = 0; i < b->n; ++i) {
        b->host_desc[i].step = 0;
        max_L = std::max(max_L, b->L[i]);
    }
    PGG_BCUDA(cudaMemcpyAsync(b->desc_d, b->host_desc.data(), size_t(b->n) * sizeof(ReplicaDesc), cudaMemcpyHostToDevice, b->stream));
    // one launch for all replicas, from the descriptors just uploaded
    const uint64_t max_words = static_cast<uint64_t>(max_L) * max_L / 32;
    const unsigned gx = static_cast<unsigned>(std::min<uint64_t>((max_words + 255) / 256, 1024));
    const unsigned gy = static_cast<unsigned>(std::min(b->n, 65535));
    pgg::k_batch_init<<<dim3(gx, gy), 256, 0, b->stream>>>(b->desc_d, b->n, thr);
    PGG_BCUDA(cudaGetLastError());
    PGG_BCUDA(cudaStreamSynchronize(b->stream));
    return PGG_OK;
}

int pgg_batch_set_team_warps(pgg_batch *b, const int *warps) {
    pgg::clear_error();
    if (!b || !warps) return bfail(PGG_ERR_ARG, "pgg_batch_set_team_warps: NULL argument");
    for (int c = 0; c < pgg::kSizeClasses; ++c) {
        const int w = warps[c];
        if (w != 1 && w != 2 && w != 4 && w != 8 && w != 16 && w != 32)
            return bfail(PGG_ERR_ARG, "pgg_batch_set_team_warps: warps per replica must be 1, 2, 4, 8, 16 or 32");
    }
    for (int c = 0; c < pgg::kSizeClasses; ++c)
        if (warps[c] > b->cta_threads / 32)
            return bfail(PGG_ERR_ARG, "pgg_batch_set_team_warps: %d warps exceed the %d-thread CTA", warps[c], b->cta_threads);
    std::memcpy(b->team_warps, warps, sizeof b->team_warps);
    b->jobs_valid = false;
    return PGG_OK;
}

int pgg_batch_set_cta_threads(pgg_batch *b, int threads) {
    pgg::clear_error();
    if (!b) return bfail(PGG_ERR_ARG, "pgg_batch_set_cta_threads: NULL batch");
    if (threads != 512 && threads != 1024) return bfail(PGG_ERR_ARG, "pgg_batch_set_cta_threads: 512 or 1024");
    b->cta_threads = threads;
    for (int c = 0; c < pgg::kSizeClasses; ++c)
        if (b->team_warps[c] > threads / 32) b->team_warps[c] = threads / 32;
    b->jobs_valid = false;
    return PGG_OK;
}

int pgg_batch_get_cta_threads(const pgg_batch *b, int *threads) {
    pgg::clear_error();
    if (!b || !threads) return bfail(PGG_ERR_ARG, "pgg_batch_get_cta_threads: NULL argument");
    *threads = b->cta_threads;
    return PGG_OK;
}

int pgg_batch_get_team_warps(const pgg_batch *b, int *warps) {
    pgg::clear_error();
    if (!b || !warps) return bfail(PGG_ERR_ARG, "pgg_batch_get_team_warps: NULL argument");
    std::memcpy(warps, b->team_warps, sizeof b->team_warps);
    return PGG_OK;
}

int pgg_batch_step_mcs(pgg_batch *b, int n_mcs, uint32_t *counts) {
    pgg::clear_error();
    if (!b) return bfail(PGG_ERR_ARG, "pgg_batch_step_mcs: NULL batch");
    if (n_mcs < 0) return bfail(PGG_ERR_ARG, "pgg_batch_step_mcs: n_mcs < 0");
    if (n_mcs == 0) return PGG_OK;
    // every replica's step + 16 n_mcs stays below 2^56 (n_mcs < 2^31, so 16 n_mcs cannot wrap)
    for (int i = 0; i < b->n; ++i)
        if (b->host_desc[i].step > (1ull << 56) - 1 - 16ull * static_cast<uint64_t>(n_mcs))
            return bfail(PGG_ERR_ARG, "pgg_batch_step_mcs: replica %d: step counter would pass 2^56", i);
    PGG_BCUDA(cudaSetDevice(b->device));
    if (!b->jobs_valid) {
        int rc = build_jobs(b);
        if (rc) return rc;
    }
    const int64_t need = int64_t(b->n) * n_mcs;
    if (counts && need > b->counts_cap) {
        if (b->counts_d) cudaFree(b->counts_d);
        b->counts_d = nullptr;
        b->counts_cap = 0;
        cudaError_t e = cudaMalloc(&b->counts_d, size_t(need) * sizeof(uint32_t));
        if (e != cudaSuccess) return bfail(PGG_ERR_OOM, "pgg_batch_step_mcs: counts: %s", cudaGetErrorString(e));
        b->counts_cap = need;
        drop_graph(b);
    }
    if (!b->use_graph) {
        PGG_BCUDA(enqueue_launch(b, n_mcs, counts != nullptr, b->stream));
    } else {
        // one persistent launch captured once per (n_mcs, counts) and replayed: the replicas'
        // state lives in device descriptors, so every replay continues from the last one
        if (b->graph_n_mcs != n_mcs || b->graph_counts != (counts != nullptr) || !b->graph_exec) {
            drop_graph(b);
            if (!b->capture_stream) PGG_BCUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
            PGG_BCUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue_launch(b, n_mcs, counts != nullptr, b->capture_stream);
            cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &b->graph);
            if (e != cudaSuccess || e2 != cudaSuccess)
                return bfail(PGG_ERR_CUDA, "pgg_batch_step_mcs: graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
            PGG_BCUDA(cudaGraphInstantiate(&b->graph_exec, b->graph, 0));
            b->graph_n_mcs = n_mcs;
            b->graph_counts = counts != nullptr;
        }
        PGG_BCUDA(cudaGraphLaunch(b->graph_exec, b->stream));
    }
    for (int i = 0; i < b->n; ++i) b->host_desc[i].step += 16ull * static_cast<uint64_t>(n_mcs);
    if (counts) {
        cudaPointerAttributes attr;
        bool dev = cudaPointerGetAttributes(&attr, counts) == cudaSuccess &&
                   (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        PGG_BCUDA(cudaMemcpyAsync(counts, b->counts_d, size_t(need) * sizeof(uint32_t),
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
        if (!dev) PGG_BCUDA(cudaStreamSynchronize(b->stream));
    }
    return PGG_OK;
}

int pgg_batch_get_lattice(pgg_batch *b, int i, uint8_t *host_out, uint64_t *step_out) {
    pgg::clear_error();
    if (!b || !host_out || i < 0 || i >= b->n) return bfail(PGG_ERR_ARG, "pgg_batch_get_lattice: bad argument");
    PGG_BCUDA(cudaSetDevice(b->device));
    const int L = b->L[i];
    std::vector<uint32_t> words(lattice_words(L));
    PGG_BCUDA(cudaMemcpyAsync(words.data(), b->host_desc[i].lat, words.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream));
    PGG_BCUDA(cudaStreamSynchronize(b->stream));
    for (size_t x = 0; x < size_t(L) * L; ++x) host_out[x] = static_cast<uint8_t>((words[x >> 5] >> (x & 31)) & 1u);
    if (step_out) *step_out = b->host_desc[i].step;
    return PGG_OK;
}

int pgg_batch_set_lattice(pgg_batch *b, int i, const uint8_t *host_in, uint64_t step) {
    pgg::clear_error();
    if (!b || !host_in || i < 0 || i >= b->n) return bfail(PGG_ERR_ARG, "pgg_batch_set_lattice: bad argument");
    if (step >= (1ull << 56)) return bfail(PGG_ERR_ARG, "pgg_batch_set_lattice: step >= 2^56");
    PGG_BCUDA(cudaSetDevice(b->device));
    const int L = b->L[i];
    std::vector<uint32_t> words(lattice_words(L), 0u);
    for (size_t x = 0; x < size_t(L) * L; ++x)
        if (host_in[x]) words[x >> 5] |= 1u << (x & 31);
    b->host_desc[i].step = step;
    PGG_BCUDA(cudaMemcpyAsync(b->host_desc[i].lat, words.data(), words.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, b->stream));
    PGG_BCUDA(cudaMemcpyAsync(b->desc_d + i, &b->host_desc[i], sizeof(ReplicaDesc), cudaMemcpyHostToDevice, b->stream));
    PGG_BCUDA(cudaStreamSynchronize(b->stream));
    return PGG_OK;
}

int pgg_batch_size(const pgg_batch *b, int *n) {
    pgg::clear_error();
    if (!b || !n) return bfail(PGG_ERR_ARG, "pgg_batch_size: NULL argument");
    *n = b->n;
    return PGG_OK;
}

int pgg_batch_use_graph(pgg_batch *b, int enable) {
    pgg::clear_error();
    if (!b) return bfail(PGG_ERR_ARG, "pgg_batch_use_graph: NULL batch");
    b->use_graph = enable != 0;
    return PGG_OK;
}

int pgg_batch_autotune(pgg_batch *b, int n_mcs, int *warps_out, float *ms_out) {
    pgg::clear_error();
    if (!b) return bfail(PGG_ERR_ARG, "pgg_batch_autotune: NULL batch");
    if (n_mcs < 1 || n_mcs > 10000) return bfail(PGG_ERR_ARG, "pgg_batch_autotune: n_mcs in [1, 10000]");
    PGG_BCUDA(cudaSetDevice(b->device));
    struct Cand { int cta; int w[pgg::kSizeClasses]; };
    const Cand cands[] = {
        {1024, {1, 1, 2, 8, 32}}, {1024, {1, 1, 2, 4, 16}}, {1024, {1, 2, 4, 16, 32}}, {1024, {1, 1, 1, 4, 32}},
        {512, {1, 1, 2, 8, 16}},  {512, {1, 1, 2, 4, 16}},  {512, {1, 2, 4, 8, 16}},   {512, {1, 1, 1, 4, 8}},
    };
    size_t total_words = 0;
    for (int i = 0; i < b->n; ++i) total_words += lattice_words(b->L[i]);
    uint32_t *saved = nullptr;
    cudaError_t e = cudaMalloc(&saved, total_words * sizeof(uint32_t));
    if (e != cudaSuccess) return bfail(PGG_ERR_OOM, "pgg_batch_autotune: %s", cudaGetErrorString(e));
    std::vector<ReplicaDesc> desc0 = b->host_desc;
    const int cta0 = b->cta_threads;
    int w0[pgg::kSizeClasses];
    std::memcpy(w0, b->team_warps, sizeof w0);
    const bool g0 = b->use_graph;
    b->use_graph = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int rc = PGG_OK;
    float best_ms = 1e30f;
    Cand best = {cta0, {w0[0], w0[1], w0[2], w0[3], w0[4]}};
    if ((e = cudaEventCreate(&ev0)) != cudaSuccess || (e = cudaEventCreate(&ev1)) != cudaSuccess ||
        (e = cudaMemcpyAsync(saved, b->lat_pool, total_words * sizeof(uint32_t), cudaMemcpyDeviceToDevice, b->stream)) != cudaSuccess)
        rc = bfail(PGG_ERR_CUDA, "pgg_batch_autotune: %s", cudaGetErrorString(e));
    for (const Cand &c : cands) {
        if (rc) break;
        b->cta_threads = c.cta;
        std::memcpy(b->team_warps, c.w, sizeof c.w);
        b->jobs_valid = false;
        float ms = 0;
        for (int rep = 0; rep < 2 && rc == PGG_OK; ++rep) {
            b->host_desc = desc0;
            if ((e = cudaMemcpyAsync(b->lat_pool, saved, total_words * sizeof(uint32_t), cudaMemcpyDeviceToDevice, b->stream)) != cudaSuccess ||
                (e = cudaMemcpyAsync(b->desc_d, b->host_desc.data(), size_t(b->n) * sizeof(ReplicaDesc), cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
                (e = cudaEventRecord(ev0, b->stream)) != cudaSuccess) {
                rc = bfail(PGG_ERR_CUDA, "pgg_batch_autotune: %s", cudaGetErrorString(e));
                break;
            }
            rc = pgg_batch_step_mcs(b, n_mcs, nullptr);
            if (rc) break;
            if ((e = cudaEventRecord(ev1, b->stream)) != cudaSuccess || (e = cudaEventSynchronize(ev1)) != cudaSuccess ||
                (e = cudaEventElapsedTime(&ms, ev0, ev1)) != cudaSuccess)
                rc = bfail(PGG_ERR_CUDA, "pgg_batch_autotune: timing: %s", cudaGetErrorString(e));
        }
        if (rc == PGG_OK && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    // restore replicas; keep the winner
    b->host_desc = desc0;
    cudaMemcpyAsync(b->lat_pool, saved, total_words * sizeof(uint32_t), cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(b->desc_d, b->host_desc.data(), size_t(b->n) * sizeof(ReplicaDesc), cudaMemcpyHostToDevice, b->stream);
    cudaStreamSynchronize(b->stream);
    cudaFree(saved);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    b->use_graph = g0;
    if (rc) {
        b->cta_threads = cta0;
        std::memcpy(b->team_warps, w0, sizeof w0);
        b->jobs_valid = false;
        return rc;
    }
    b->cta_threads = best.cta;
    std::memcpy(b->team_warps, best.w, sizeof best.w);
    b->jobs_valid = false;
    drop_graph(b);
    if (warps_out) std::memcpy(warps_out, best.w, sizeof best.w);
    if (ms_out) *ms_out = best_ms;
    return PGG_OK;
}

void pgg_batch_destroy(pgg_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->desc_d) cudaFree(b->desc_d);
    if (b->lat_pool) cudaFree(b->lat_pool);
    if (b->table_pool) cudaFree(b->table_pool);
    if (b->members_d) cudaFree(b->members_d);
    if (b->jobs_d) cudaFree(b->jobs_d);
    if (b->counter_d) cudaFree(b->counter_d);
    if (b->counts_d) cudaFree(b->counts_d);
    drop_graph(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    delete b;
}

}  // extern "C"
