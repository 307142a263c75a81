// pgg_abi.cu -- the C ABI declared in include/pgg.h: context management, the host-built
// adoption threshold table of Eq. (3), and the scheduling of the step kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "pgg.h"
#include "pgg_device.cuh"
#include "pgg_internal.h"

namespace pgg {

// Adoption thresholds of Eq. (3) for every (s_x, S_x, S_y) with s_y = 1 - s_x:
// P(s, S) = (r S)/5 - 5 s is the payoff summed over a player's five groups (Eq. (1)-(2),
// c = 1, G = 5); W = 1 / (1 + exp((P_x - P_y) / K)); T = floor(W 2^32), 2^32 - 1 if W >= 1.
// Evaluated in IEEE double precision with the host libm (compiled without contraction).
void build_threshold_table(double r, double K, uint32_t *T) {
    for (int sx = 0; sx < 2; ++sx) {
        const int sy = 1 - sx;
        for (int Sx = 0; Sx < pgg::kSRange; ++Sx) {
            for (int Sy = 0; Sy < pgg::kSRange; ++Sy) {
                const double px = (r * static_cast<double>(Sx)) / 5.0 - 5.0 * static_cast<double>(sx);
                const double py = (r * static_cast<double>(Sy)) / 5.0 - 5.0 * static_cast<double>(sy);
                const double w = 1.0 / (1.0 + std::exp((px - py) / K));
                T[(sx * pgg::kSRange + Sx) * pgg::kSRange + Sy] =
                    (w >= 1.0) ? 0xFFFFFFFFu : static_cast<uint32_t>(w * 4294967296.0);
            }
        }
    }
}

// The pairwise game of Section VI: a player with n cooperating neighbours (of 4) earns
// P(s, n) = n A + (4 - n) B over its four games, (A, B) = (R, S) for a cooperator and (T, P)
// for a defector (pay = {R, S, T, P}); thresholds as above, indexed (s_x*5 + n_x)*5 + n_y.
// The rest of the 2*26*26 buffer is zero.
void build_pair_threshold_table(const double pay[4], double K, uint32_t *T) {
    std::memset(T, 0, sizeof(uint32_t) * pgg::kTableEntries);
    for (int sx = 0; sx < 2; ++sx) {
        const int sy = 1 - sx;
        for (int nx = 0; nx < pgg::kNRange; ++nx) {
            for (int ny = 0; ny < pgg::kNRange; ++ny) {
                const double ax = sx ? pay[0] : pay[2], bx = sx ? pay[1] : pay[3];
                const double ay = sy ? pay[0] : pay[2], by = sy ? pay[1] : pay[3];
                const double px = static_cast<double>(nx) * ax + static_cast<double>(4 - nx) * bx;
                const double py = static_cast<double>(ny) * ay + static_cast<double>(4 - ny) * by;
                const double w = 1.0 / (1.0 + std::exp((px - py) / K));
                T[(sx * pgg::kNRange + nx) * pgg::kNRange + ny] =
                    (w >= 1.0) ? 0xFFFFFFFFu : static_cast<uint32_t>(w * 4294967296.0);
            }
        }
    }
}

}  // namespace pgg

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define PGG_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail(PGG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr uint64_t kMaxStep = (1ull << 56);

bool is_pow2_fuse(int k) { return k == 1 || k == 2 || k == 4 || k == 8 || k == 16; }

}  // namespace

namespace pgg {

int record_error(int code, const char *message) {
    g_last_error = message;
    return code;
}

void clear_error() { g_last_error.clear(); }

}  // namespace pgg

struct pgg_ctx {
    int L = 0;
    double r = 0, K = 0;
    int game = PGG_GAME_GROUP;              // pgg_game
    double pay[4] = {0.0, 0.0, 0.0, 0.0};   // pairwise payoff matrix {R, S, T, P}
    int layout = PGG_U8;
    cudaStream_t stream = nullptr;
    int device = 0;
    uint64_t seed = 0;
    uint64_t step = 0;
    void *lat = nullptr;      // current lattice
    void *lat_alt = nullptr;  // second buffer for fused (k > 1) launches
    size_t lat_bytes = 0;
    uint32_t *table_d = nullptr;
    uint32_t table_h[pgg::kTableEntries];
    unsigned long long *counts_d = nullptr;
    int64_t counts_cap = 0;
    uint8_t *staging_d = nullptr;  // L*L bytes for uint8 <-> bit-packed transfers
    int kernel = PGG_KERNEL_AUTO;
    int k_fuse = 1;
    int tile_x = 0, tile_y = 0;
    unsigned long long *running_d = nullptr;  // cooperator count carried by the direct kernel
    bool running_valid = false;               // running_d equals the lattice's count
    // resident kernel
    int sms = 0;
    size_t smem_optin = 0;
    uint32_t *mailbox_d = nullptr;
    unsigned int *ctr_d = nullptr;
    unsigned int ctr_launches = 0;  // resident launches since ctr_d was last zeroed
    // the resident kernel's per-MCS count slots: kResidentCountSlots sums, then as many tallies;
    // zero between launches, except after a launch that stopped on a time-out
    unsigned long long *count_slots_d = nullptr;
    bool count_slots_dirty = true;
    // the lattice's column-class copy, kept by resident launches that use it (L*L/32 words); valid
    // while nothing else has written the lattice since (cleared wherever running_valid is)
    uint32_t *cls_d = nullptr;
    bool cls_valid = false;
    int *status_d = nullptr;
    int *status_h = nullptr;                  // pinned: the status word read back with the counts
    unsigned long long *counts_h = nullptr;   // pinned: counts on their way to a host buffer
    int64_t counts_h_cap = 0;
    unsigned int spin_limit = 1u << 22;
    // overlapped upload (pgg_stage_lattice_packed): two bit-packed buffers filled by a copy
    // stream of the context's own while the context stream computes
    cudaStream_t copy_stream = nullptr;
    uint32_t *stage_d[2] = {nullptr, nullptr};
    cudaEvent_t stage_ready[2] = {nullptr, nullptr};  // the copy into stage_d[b] has completed
    cudaEvent_t stage_free[2] = {nullptr, nullptr};   // the context stream no longer uses stage_d[b]
    int stage_next = 0;        // buffer the next pgg_stage_lattice_packed fills
    int stage_pending = -1;    // buffer holding a staged lattice not yet applied, or -1
    uint64_t stage_step = 0;   // step counter that comes with the staged lattice
    // kernel timing (pgg_set_kernel_timing): an event pair around every step-kernel launch
    bool timing = false;
    std::vector<cudaEvent_t> tev_start, tev_stop;
    size_t tev_used = 0;
};

namespace {

// Resolved schedule: (kernel, k, tile_x, tile_y).
struct Schedule {
    int kernel, k, tile_x, tile_y;
};

bool tiled_supported(const pgg_ctx *c) { return c->L >= 64 && c->L % 64 == 0; }

// Schedules chosen by pgg_autotune, per (device, L, layout, game); consulted by
// PGG_KERNEL_AUTO.
std::mutex g_tuned_mutex;
std::map<std::tuple<int, int, int, int>, Schedule> g_tuned;

bool tuned_lookup(const pgg_ctx *c, Schedule *out) {
    std::lock_guard<std::mutex> lock(g_tuned_mutex);
    auto it = g_tuned.find(std::make_tuple(c->device, c->L, c->layout, c->game));
    if (it == g_tuned.end()) return false;
    *out = it->second;
    return true;
}

Schedule resolve_schedule(const pgg_ctx *c) {
    Schedule s{c->kernel, c->k_fuse, c->tile_x, c->tile_y};
    if (s.kernel == PGG_KERNEL_AUTO) tuned_lookup(c, &s);  // then resolved like an explicit choice
    if (s.kernel == PGG_KERNEL_AUTO) {
        if (c->L >= 2048 && pgg::resident_bands(c->layout, c->L, c->sms, c->smem_optin) > 0) {
            s = {PGG_KERNEL_RESIDENT, 16, 0, 0};
        } else if (pgg::direct_supported(c->layout, c->L)) {
            s = {PGG_KERNEL_DIRECT, 1, 8, 256};
        } else if (!tiled_supported(c)) {
            s = {PGG_KERNEL_SIMPLE, 1, 0, 0};
        } else {
            s.kernel = PGG_KERNEL_TILED;
            s.k = 1;
            s.tile_x = 0;
            s.tile_y = 0;
        }
    }
    if (s.kernel == PGG_KERNEL_RESIDENT) {
        s.k = 16;
        s.tile_x = pgg::resident_bands(c->layout, c->L, c->sms, c->smem_optin);
        // tile_y: sublattice steps per halo exchange (1, 2 or 4), the largest that fits by default
        const int smax = s.tile_x > 0 ? pgg::resident_max_steps_per_exchange(c->L, s.tile_x, c->smem_optin) : 1;
        if (s.tile_y != 1 && s.tile_y != 2 && s.tile_y != 4) s.tile_y = smax;
        if (s.tile_y > smax) s.tile_y = smax;
        return s;
    }
    if (s.kernel == PGG_KERNEL_DIRECT) {
        s.k = 1;
        if (s.tile_x != 4 && s.tile_x != 8) s.tile_x = 8;
        if (s.tile_y != 64 && s.tile_y != 128 && s.tile_y != 256) s.tile_y = 256;
        return s;
    }
    if (s.kernel == PGG_KERNEL_TILED) {
        if (s.tile_x <= 0) s.tile_x = c->L >= 1024 ? 1024 : c->L;
        if (s.tile_y <= 0) s.tile_y = c->L >= 64 ? 64 : c->L;
        if (s.tile_x > c->L) s.tile_x = c->L;
        if (s.tile_y > c->L) s.tile_y = c->L;
    } else {
        s.k = 1;
        s.tile_x = s.tile_y = 0;
    }
    return s;
}

int ensure_counts(pgg_ctx *c, int64_t n) {
    if (n <= c->counts_cap) return PGG_OK;
    int64_t cap = c->counts_cap > 0 ? c->counts_cap : 1024;
    while (cap < n) cap *= 2;
    if (c->counts_d) cudaFree(c->counts_d);
    c->counts_d = nullptr;
    c->counts_cap = 0;
    cudaError_t e = cudaMalloc(&c->counts_d, static_cast<size_t>(cap) * sizeof(unsigned long long));
    if (e != cudaSuccess) return fail(PGG_ERR_OOM, "cudaMalloc(counts, %lld): %s", (long long)cap, cudaGetErrorString(e));
    c->counts_cap = cap;
    return PGG_OK;
}

int ensure_alt(pgg_ctx *c) {
    if (c->lat_alt) return PGG_OK;
    cudaError_t e = cudaMalloc(&c->lat_alt, c->lat_bytes);
    if (e != cudaSuccess) return fail(PGG_ERR_OOM, "cudaMalloc(second lattice buffer): %s", cudaGetErrorString(e));
    return PGG_OK;
}

int ensure_staging(pgg_ctx *c) {
    if (c->staging_d) return PGG_OK;
    cudaError_t e = cudaMalloc(&c->staging_d, static_cast<size_t>(c->L) * c->L);
    if (e != cudaSuccess) return fail(PGG_ERR_OOM, "cudaMalloc(staging): %s", cudaGetErrorString(e));
    return PGG_OK;
}

// Release the overlapped-upload resources (after the copy stream has drained).
void release_stage(pgg_ctx *c) {
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
        c->copy_stream = nullptr;
    }
    for (int b = 0; b < 2; ++b) {
        if (c->stage_d[b]) cudaFree(c->stage_d[b]);
        if (c->stage_ready[b]) cudaEventDestroy(c->stage_ready[b]);
        if (c->stage_free[b]) cudaEventDestroy(c->stage_free[b]);
        c->stage_d[b] = nullptr;
        c->stage_ready[b] = c->stage_free[b] = nullptr;
    }
    c->stage_next = 0;
    c->stage_pending = -1;
}

// The copy stream, both staging buffers and their events, all or none (a partial failure
// releases what was made, so a later call starts afresh).
int ensure_stage(pgg_ctx *c) {
    if (c->copy_stream) return PGG_OK;
    const size_t bytes = static_cast<size_t>(c->L) * c->L / 8;
    cudaError_t e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) c->copy_stream = nullptr;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        if ((e = cudaMalloc(&c->stage_d[b], bytes)) != cudaSuccess) { c->stage_d[b] = nullptr; break; }
        if ((e = cudaEventCreateWithFlags(&c->stage_ready[b], cudaEventDisableTiming)) != cudaSuccess) {
            c->stage_ready[b] = nullptr;
            break;
        }
        if ((e = cudaEventCreateWithFlags(&c->stage_free[b], cudaEventDisableTiming)) != cudaSuccess) {
            c->stage_free[b] = nullptr;
            break;
        }
        e = cudaEventRecord(c->stage_free[b], c->stream);  // both buffers start free
    }
    if (e != cudaSuccess) {
        release_stage(c);
        return fail(e == cudaErrorMemoryAllocation ? PGG_ERR_OOM : PGG_ERR_CUDA,
                    "pgg_stage_lattice_packed: copy stream, buffers or events: %s", cudaGetErrorString(e));
    }
    return PGG_OK;
}

// Make a staged lattice the context's lattice, in stream order: the context stream waits for
// its copy; a bit-packed context then takes the staged buffer as its lattice and hands its old
// lattice buffer to the stage slot (no copy), a uint8 context unpacks the staged words into its
// lattice. The event recorded after that frees the slot's buffer for a later stage call once all
// work queued so far (which may still read the old lattice) has run. Every entry point that reads
// or writes the lattice or the step counter calls this first.
int apply_stage(pgg_ctx *c) {
    const int b = c->stage_pending;
    if (b < 0) return PGG_OK;
    c->stage_pending = -1;
    PGG_CUDA(cudaStreamWaitEvent(c->stream, c->stage_ready[b], 0));
    if (c->layout == PGG_BITPACK) {
        void *old = c->lat;
        c->lat = c->stage_d[b];
        c->stage_d[b] = static_cast<uint32_t *>(old);
    } else {
        PGG_CUDA(pgg::launch_unpack(c->stage_d[b], static_cast<uint8_t *>(c->lat), c->L, c->stream));
    }
    PGG_CUDA(cudaEventRecord(c->stage_free[b], c->stream));
    c->step = c->stage_step;
    c->running_valid = false;
    c->cls_valid = false;
    return PGG_OK;
}

// Event before a step-kernel launch when kernel timing is on (pgg_set_kernel_timing).
int timing_start(pgg_ctx *c) {
    if (!c->timing) return PGG_OK;
    if (c->tev_used == c->tev_start.size()) {
        cudaEvent_t a = nullptr, b = nullptr;
        cudaError_t e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        if (e != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            return fail(PGG_ERR_CUDA, "kernel timing: cudaEventCreate: %s", cudaGetErrorString(e));
        }
        c->tev_start.push_back(a);
        c->tev_stop.push_back(b);
    }
    PGG_CUDA(cudaEventRecord(c->tev_start[c->tev_used], c->stream));
    return PGG_OK;
}

// Event after that launch.
int timing_stop(pgg_ctx *c) {
    if (!c->timing) return PGG_OK;
    PGG_CUDA(cudaEventRecord(c->tev_stop[c->tev_used], c->stream));
    ++c->tev_used;
    return PGG_OK;
}

void timing_release(pgg_ctx *c) {
    for (cudaEvent_t e : c->tev_start) cudaEventDestroy(e);
    for (cudaEvent_t e : c->tev_stop) cudaEventDestroy(e);
    c->tev_start.clear();
    c->tev_stop.clear();
    c->tev_used = 0;
}

// Report (and clear) a bounded wait that ran out in an earlier resident launch.
int status_result(pgg_ctx *c, int st) {
    if (st) {
        c->count_slots_dirty = true;  // a stopped resident launch may have left count slots in use
        PGG_CUDA(cudaMemsetAsync(c->status_d, 0, sizeof(int), c->stream));
        PGG_CUDA(cudaStreamSynchronize(c->stream));
        c->running_valid = false;
        c->cls_valid = false;
        if (st & 8)
            return fail(PGG_ERR_CUDA, "a resident-kernel CTA stopped after a time-out while a halo copy into its "
                                      "shared memory was still unconfirmed; results on this device are undefined: "
                                      "destroy the context and reset the device's CUDA context");
        if (st & 4)
            return fail(PGG_ERR_STATE, "an index check of the checked build failed: a kernel computed an address "
                                       "outside its buffer (the access was skipped; the lattice is not a valid state)");
        if (st & 2)
            return fail(PGG_ERR_CUDA, "the resident kernel found its shared rows or the mailbox not 16-byte aligned "
                                      "and did not run; the lattice is unchanged");
        return fail(PGG_ERR_TIMEOUT,
                    "a resident-kernel CTA waited longer than %u polls for a neighbour; the lattice is not "
                    "a valid state (restore it with pgg_set_lattice or pgg_seed)",
                    c->spin_limit);
    }
    return PGG_OK;
}

int check_status(pgg_ctx *c) {
    PGG_CUDA(cudaMemcpyAsync(c->status_h, c->status_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PGG_CUDA(cudaStreamSynchronize(c->stream));
    return status_result(c, *c->status_h);
}

bool is_device_pointer(const void *p);

// Hand the n counts of a pgg_step_mcs call to the caller. Device memory is filled
// asynchronously. Host memory is filled through a pinned buffer, with the status word read
// back by the same synchronisation, so that a failed bounded wait or index check is reported by
// this call.
int deliver_counts(pgg_ctx *c, uint64_t *out, int64_t n) {
    const size_t bytes = static_cast<size_t>(n) * sizeof(uint64_t);
    if (is_device_pointer(out)) {
        PGG_CUDA(cudaMemcpyAsync(out, c->counts_d, bytes, cudaMemcpyDeviceToDevice, c->stream));
        return PGG_OK;
    }
    if (n > c->counts_h_cap) {
        int64_t cap = c->counts_h_cap > 0 ? c->counts_h_cap : 1024;
        while (cap < n) cap *= 2;
        if (c->counts_h) cudaFreeHost(c->counts_h);
        c->counts_h = nullptr;
        c->counts_h_cap = 0;
        cudaError_t e = cudaMallocHost(&c->counts_h, static_cast<size_t>(cap) * sizeof(unsigned long long));
        if (e != cudaSuccess) return fail(PGG_ERR_OOM, "cudaMallocHost(counts, %lld): %s", (long long)cap, cudaGetErrorString(e));
        c->counts_h_cap = cap;
    }
    PGG_CUDA(cudaMemcpyAsync(c->counts_h, c->counts_d, bytes, cudaMemcpyDeviceToHost, c->stream));
    PGG_CUDA(cudaMemcpyAsync(c->status_h, c->status_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PGG_CUDA(cudaStreamSynchronize(c->stream));
    std::memcpy(out, c->counts_h, bytes);
    return status_result(c, *c->status_h);
}

// Rebuild the host table for the context's game and parameters and copy it to the device.
int upload_table(pgg_ctx *c) {
    if (c->game == PGG_GAME_PAIRWISE) pgg::build_pair_threshold_table(c->pay, c->K, c->table_h);
    else pgg::build_threshold_table(c->r, c->K, c->table_h);
    // the host table is copied by value before the call returns
    PGG_CUDA(cudaMemcpyAsync(c->table_d, c->table_h, sizeof c->table_h, cudaMemcpyHostToDevice, c->stream));
    PGG_CUDA(cudaStreamSynchronize(c->stream));
    return PGG_OK;
}

bool is_device_pointer(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

const char *pgg_last_error(void) { return g_last_error.c_str(); }

const char *pgg_version(void) { return "pgg-gb300 0.1 (sm_103a)"; }

int pgg_create(pgg_ctx **out, int L, double r, double K, int layout, void *cuda_stream) {
    g_last_error.clear();
    if (!out) return fail(PGG_ERR_ARG, "pgg_create: out is NULL");
    *out = nullptr;
    if (layout != PGG_U8 && layout != PGG_BITPACK) return fail(PGG_ERR_ARG, "pgg_create: unknown layout %d", layout);
    if (L < 4 || L > 32768 || L % 4 != 0)
        return fail(PGG_ERR_ARG, "pgg_create: L = %d must be a multiple of 4 in [4, 32768]", L);
    if (layout == PGG_BITPACK && L % 32 != 0)
        return fail(PGG_ERR_ARG, "pgg_create: bit-packed lattices need L %% 32 == 0 (L = %d)", L);
    if (!(r > 0.0) || !std::isfinite(r)) return fail(PGG_ERR_ARG, "pgg_create: r must be > 0");
    if (!(K > 0.0) || !std::isfinite(K)) return fail(PGG_ERR_ARG, "pgg_create: K must be > 0");
    pgg_ctx *c = new (std::nothrow) pgg_ctx();
    if (!c) return fail(PGG_ERR_OOM, "pgg_create: host allocation failed");
    c->L = L;
    c->r = r;
    c->K = K;
    c->layout = layout;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return fail(PGG_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    {
        int sms = 0, optin = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) == cudaSuccess) {
            c->sms = sms;
            c->smem_optin = static_cast<size_t>(optin) > 2048 ? static_cast<size_t>(optin) - 2048 : 0;
        }
    }
    const uint64_t sites = static_cast<uint64_t>(L) * L;
    c->lat_bytes = layout == PGG_U8 ? sites : sites / 8;
    pgg::build_threshold_table(r, K, c->table_h);
    if ((e = cudaMalloc(&c->lat, c->lat_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&c->table_d, sizeof c->table_h)) != cudaSuccess ||
        (e = cudaMalloc(&c->status_d, sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost(&c->status_h, sizeof(int))) != cudaSuccess) {
        pgg_destroy(c);
        return fail(PGG_ERR_OOM, "pgg_create: cudaMalloc: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(c->table_d, c->table_h, sizeof c->table_h, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->lat, 0, c->lat_bytes, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->status_d, 0, sizeof(int), c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
        pgg_destroy(c);
        return fail(PGG_ERR_CUDA, "pgg_create: %s", cudaGetErrorString(e));
    }
    *out = c;
    return PGG_OK;
}

int pgg_set_params(pgg_ctx *c, double r, double K) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_set_params: NULL context");
    if (!(r > 0.0) || !std::isfinite(r) || !(K > 0.0) || !std::isfinite(K))
        return fail(PGG_ERR_ARG, "pgg_set_params: need r > 0 and K > 0");
    PGG_CUDA(cudaSetDevice(c->device));
    c->r = r;
    c->K = K;
    return upload_table(c);
}

int pgg_set_game(pgg_ctx *c, int game, const double payoff[4]) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_set_game: NULL context");
    if (game != PGG_GAME_GROUP && game != PGG_GAME_PAIRWISE) return fail(PGG_ERR_ARG, "pgg_set_game: unknown game %d", game);
    if (game == PGG_GAME_PAIRWISE) {
        if (!payoff) return fail(PGG_ERR_ARG, "pgg_set_game: the pairwise game needs its payoff matrix");
        for (int q = 0; q < 4; ++q)
            if (!std::isfinite(payoff[q])) return fail(PGG_ERR_ARG, "pgg_set_game: payoff[%d] is not finite", q);
    }
    PGG_CUDA(cudaSetDevice(c->device));
    c->game = game;
    for (int q = 0; q < 4; ++q) c->pay[q] = game == PGG_GAME_PAIRWISE ? payoff[q] : 0.0;
    return upload_table(c);
}

int pgg_get_game(const pgg_ctx *c, int *game, double *payoff_out) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_get_game: NULL context");
    if (game) *game = c->game;
    if (payoff_out)
        for (int q = 0; q < 4; ++q) payoff_out[q] = c->pay[q];
    return PGG_OK;
}

int pgg_seed(pgg_ctx *c, uint64_t seed, double p) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_seed: NULL context");
    if (!(p >= 0.0 && p <= 1.0)) return fail(PGG_ERR_ARG, "pgg_seed: p must be in [0, 1]");
    PGG_CUDA(cudaSetDevice(c->device));
    if (int rc_stage = apply_stage(c)) return rc_stage;
    uint64_t thr = p >= 1.0 ? (1ull << 32) : static_cast<uint64_t>(p * 4294967296.0);
    PGG_CUDA(pgg::launch_init(c->layout, c->lat, c->L, seed, thr, c->stream));
    c->seed = seed;
    c->step = 0;
    c->running_valid = false;
    c->cls_valid = false;
    return PGG_OK;
}

int pgg_step_mcs(pgg_ctx *c, int64_t n_mcs, uint64_t *coop_per_mcs) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_step_mcs: NULL context");
    if (n_mcs < 0) return fail(PGG_ERR_ARG, "pgg_step_mcs: n_mcs < 0");
    if (n_mcs == 0) return PGG_OK;
    const uint64_t step_in = c->stage_pending >= 0 ? c->stage_step : c->step;
    // step_in + 16 n_mcs < 2^56 (step_in < 2^56 always), tested without forming the sum
    if (static_cast<uint64_t>(n_mcs) > (kMaxStep - 1 - step_in) / 16)
        return fail(PGG_ERR_ARG, "pgg_step_mcs: step counter would pass 2^56");
    PGG_CUDA(cudaSetDevice(c->device));
    if (int rc_stage = apply_stage(c)) return rc_stage;
    int rc = ensure_counts(c, n_mcs);
    if (rc) return rc;
    const Schedule s = resolve_schedule(c);
    if (s.kernel == PGG_KERNEL_TILED && s.k > 1 && (rc = ensure_alt(c))) return rc;
    if (s.kernel == PGG_KERNEL_RESIDENT) {
        const int bands = s.tile_x;
        if (bands < 1) return fail(PGG_ERR_STATE, "pgg_step_mcs: the lattice cannot be resident");
        const size_t mb_words = pgg::resident_mailbox_words(c->L, bands);
        if (!c->mailbox_d) {
            // the mailbox, then one word per band that the kernel keeps between launches
            cudaError_t e = cudaMalloc(&c->mailbox_d, (mb_words + bands) * sizeof(uint32_t));
            if (e == cudaSuccess) e = cudaMalloc(&c->ctr_d, sizeof(unsigned int) * bands);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->mailbox_d + mb_words, 0, sizeof(uint32_t) * bands, c->stream);
            if (e == cudaSuccess)
                e = cudaMalloc(&c->count_slots_d, pgg::kResidentCountSlots * (sizeof(unsigned long long) + sizeof(unsigned int)));
            if (e != cudaSuccess) return fail(PGG_ERR_OOM, "cudaMalloc(resident buffers): %s", cudaGetErrorString(e));
        }
        // the kernel writes every count of the call itself (no memset of counts_d); its count
        // slots must be zero, which they are after every launch that ran to its end
        if (c->count_slots_dirty) {
            PGG_CUDA(cudaMemsetAsync(c->count_slots_d, 0,
                                     pgg::kResidentCountSlots * (sizeof(unsigned long long) + sizeof(unsigned int)), c->stream));
            c->count_slots_dirty = false;
        }
        // the kernel keeps the band bit-packed in shared memory; a uint8 lattice is packed as it is
        // staged and unpacked as it is written back
        pgg::ResidentArgs a;
        a.game = c->game;
        a.lat = c->layout == PGG_BITPACK ? static_cast<uint32_t *>(c->lat) : nullptr;
        a.lat8 = c->layout == PGG_U8 ? static_cast<uint8_t *>(c->lat) : nullptr;
        a.L = c->L;
        a.n_bands = bands;
        a.seed = c->seed;
        a.k0 = c->step;
        a.table = c->table_d;
        a.mailbox = c->mailbox_d;
        a.ctr = c->ctr_d;
        a.status = c->status_d;
        a.spin_limit = c->spin_limit;
        a.steps_per_exchange = s.tile_y;
        // the column-class copy makes the scan for active sites cheap; the pairwise game, whose
        // steps mostly take the dense pass, only pays for keeping it (measured at L = 8192: 0.154
        // against 0.140 ms per MCS), so it runs on the bit-packed rows alone
        a.class_copy = c->game == PGG_GAME_GROUP && pgg::resident_class_copy(c->L, bands, s.tile_y, c->smem_optin);
        if (a.class_copy && !c->cls_d) {
            // without room for it the kernel rebuilds the class copy at every launch
            if (cudaMalloc(&c->cls_d, static_cast<size_t>(c->L) * c->L / 8) != cudaSuccess) {
                c->cls_d = nullptr;
                cudaGetLastError();
            }
        }
        a.cls_g = c->cls_d;
        a.cls_load = c->cls_valid;
        a.hint = reinterpret_cast<unsigned int *>(c->mailbox_d + mb_words);
        a.count_acc = c->count_slots_d;
        a.count_tick = reinterpret_cast<unsigned int *>(c->count_slots_d + pgg::kResidentCountSlots);
        // the pass over active sites only wins for the group game up to about 10 % of a step's
        // sites adopting (measured at L = 8192); the pairwise game, whose active sites are more
        // numerous and cheaper to update whole words at a time, takes the dense pass above 1.5 %
        a.dense_per_mille = c->game == PGG_GAME_PAIRWISE ? 15u : 100u;
        // one launch covers at most 1 << 16 MCS
        for (int64_t m0 = 0; m0 < n_mcs; m0 += (1 << 16)) {
            a.n_mcs = static_cast<int>(std::min<int64_t>(n_mcs - m0, 1 << 16));
            a.counts = c->counts_d + m0;
            a.k0 = c->step;
            // a launch covers at most 2^20 steps: counters of launch n lie in [n 2^21, n 2^21 + 2^20]
            if (c->ctr_launches == 0 || c->ctr_launches >= 2047) c->ctr_launches = 0;
            a.reset_ctr = c->ctr_launches == 0;
            a.ctr_base = c->ctr_launches << 21;
            ++c->ctr_launches;
            if (int rc_t = timing_start(c)) return rc_t;
            PGG_CUDA(pgg::launch_resident(a, c->stream));
            a.cls_load = a.class_copy && a.cls_g;  // the next launch of a long call finds it there
            if (int rc_t = timing_stop(c)) return rc_t;
            c->step += 16ull * static_cast<uint64_t>(a.n_mcs);
        }
        c->running_valid = false;
        c->cls_valid = a.class_copy && a.cls_g;
        PGG_CUDA(cudaGetLastError());
        return coop_per_mcs ? deliver_counts(c, coop_per_mcs, n_mcs) : PGG_OK;
    }
    c->cls_valid = false;  // the kernels below write the lattice without its class copy
    PGG_CUDA(cudaMemsetAsync(c->counts_d, 0, static_cast<size_t>(n_mcs) * sizeof(unsigned long long), c->stream));
    if (s.kernel == PGG_KERNEL_DIRECT) {
        if (!c->running_d) {
            cudaError_t e = cudaMalloc(&c->running_d, sizeof(unsigned long long));
            if (e != cudaSuccess) return fail(PGG_ERR_OOM, "cudaMalloc(running count): %s", cudaGetErrorString(e));
            c->running_valid = false;
            c->cls_valid = false;
        }
        if (!c->running_valid) {
            PGG_CUDA(cudaMemsetAsync(c->running_d, 0, sizeof(unsigned long long), c->stream));
            PGG_CUDA(pgg::launch_popcount(c->lat, c->lat_bytes, c->running_d, c->stream));
            c->running_valid = true;
        }
    } else {
        c->running_valid = false;
        c->cls_valid = false;
    }
    for (int64_t m = 0; m < n_mcs; ++m) {
        if (s.kernel == PGG_KERNEL_DIRECT) {
            for (int j = 0; j < 16; ++j) {
                if (int rc_t = timing_start(c)) return rc_t;
                PGG_CUDA(pgg::launch_step_direct(c->game, static_cast<uint32_t *>(c->lat), c->L, c->seed, c->step, c->table_d,
                                                 c->running_d, c->status_d, s.tile_x, s.tile_y, c->stream));
                if (int rc_t = timing_stop(c)) return rc_t;
                ++c->step;
            }
            PGG_CUDA(cudaMemcpyAsync(c->counts_d + m, c->running_d, sizeof(unsigned long long),
                                     cudaMemcpyDeviceToDevice, c->stream));
        } else if (s.kernel == PGG_KERNEL_SIMPLE) {
            for (int j = 0; j < 16; ++j) {
                if (int rc_t = timing_start(c)) return rc_t;
                PGG_CUDA(pgg::launch_step_simple(c->layout, c->game, c->lat, c->L, c->seed, c->step, c->table_d, c->stream));
                if (int rc_t = timing_stop(c)) return rc_t;
                ++c->step;
            }
            PGG_CUDA(pgg::launch_popcount(c->lat, c->lat_bytes, c->counts_d + m, c->stream));
        } else {
            for (int j = 0; j < 16; j += s.k) {
                pgg::TiledArgs a;
                a.game = c->game;
                a.src = c->lat;
                a.dst = s.k == 1 ? c->lat : c->lat_alt;
                a.L = c->L;
                a.layout = c->layout;
                a.seed = c->seed;
                a.k0 = c->step;
                a.steps = s.k;
                a.tile_x = s.tile_x;
                a.tile_y = s.tile_y;
                a.table = c->table_d;
                a.count_out = (j + s.k == 16) ? c->counts_d + m : nullptr;
                a.status = c->status_d;
                if (int rc_t = timing_start(c)) return rc_t;
                PGG_CUDA(pgg::launch_step_tiled(a, c->stream));
                if (int rc_t = timing_stop(c)) return rc_t;
                if (s.k > 1) {
                    void *t = c->lat;
                    c->lat = c->lat_alt;
                    c->lat_alt = t;
                }
                c->step += s.k;
            }
        }
    }
    PGG_CUDA(cudaGetLastError());
    return coop_per_mcs ? deliver_counts(c, coop_per_mcs, n_mcs) : PGG_OK;
}

int pgg_count_coop(pgg_ctx *c, uint64_t *out) {
    g_last_error.clear();
    if (!c || !out) return fail(PGG_ERR_ARG, "pgg_count_coop: NULL argument");
    PGG_CUDA(cudaSetDevice(c->device));
    if (int rc_stage = apply_stage(c)) return rc_stage;
    int rc = ensure_counts(c, 1);
    if (rc) return rc;
    PGG_CUDA(cudaMemsetAsync(c->counts_d, 0, sizeof(unsigned long long), c->stream));
    PGG_CUDA(pgg::launch_popcount(c->lat, c->lat_bytes, c->counts_d, c->stream));
    unsigned long long v = 0;
    PGG_CUDA(cudaMemcpyAsync(&v, c->counts_d, sizeof v, cudaMemcpyDeviceToHost, c->stream));
    PGG_CUDA(cudaStreamSynchronize(c->stream));
    *out = v;
    return check_status(c);
}

int pgg_get_lattice(pgg_ctx *c, uint8_t *host_out, uint64_t *step_out) {
    g_last_error.clear();
    if (!c || !host_out) return fail(PGG_ERR_ARG, "pgg_get_lattice: NULL argument");
    PGG_CUDA(cudaSetDevice(c->device));
    if (int rc_stage = apply_stage(c)) return rc_stage;
    const size_t n = static_cast<size_t>(c->L) * c->L;
    if (c->layout == PGG_U8) {
        PGG_CUDA(cudaMemcpyAsync(host_out, c->lat, n, cudaMemcpyDeviceToHost, c->stream));
    } else {
        int rc = ensure_staging(c);
        if (rc) return rc;
        PGG_CUDA(pgg::launch_unpack(static_cast<const uint32_t *>(c->lat), c->staging_d, c->L, c->stream));
        PGG_CUDA(cudaMemcpyAsync(host_out, c->staging_d, n, cudaMemcpyDeviceToHost, c->stream));
    }
    PGG_CUDA(cudaStreamSynchronize(c->stream));
    if (step_out) *step_out = c->step;
    return check_status(c);
}

int pgg_set_lattice(pgg_ctx *c, const uint8_t *host_in, uint64_t step) {
    g_last_error.clear();
    if (!c || !host_in) return fail(PGG_ERR_ARG, "pgg_set_lattice: NULL argument");
    if (step >= kMaxStep) return fail(PGG_ERR_ARG, "pgg_set_lattice: step >= 2^56");
    PGG_CUDA(cudaSetDevice(c->device));
    if (int rc_stage = apply_stage(c)) return rc_stage;
    const size_t n = static_cast<size_t>(c->L) * c->L;
    if (c->layout == PGG_U8) {
        PGG_CUDA(cudaMemcpyAsync(c->lat, host_in, n, cudaMemcpyHostToDevice, c->stream));
        PGG_CUDA(pgg::launch_normalize(static_cast<uint8_t *>(c->lat), n, c->stream));
    } else {
        int rc = ensure_staging(c);
        if (rc) return rc;
        PGG_CUDA(cudaMemcpyAsync(c->staging_d, host_in, n, cudaMemcpyHostToDevice, c->stream));
        PGG_CUDA(pgg::launch_pack(c->staging_d, static_cast<uint32_t *>(c->lat), c->L, c->stream));
    }
    PGG_CUDA(cudaStreamSynchronize(c->stream));
    c->step = step;
    c->running_valid = false;
    c->cls_valid = false;
    return PGG_OK;
}

int pgg_get_lattice_packed(pgg_ctx *c, uint32_t *host_words_out, uint64_t *step_out) {
    g_last_error.clear();
    if (!c || !host_words_out) return fail(PGG_ERR_ARG, "pgg_get_lattice_packed: NULL argument");
    if (c->L % 32 != 0) return fail(PGG_ERR_ARG, "pgg_get_lattice_packed: needs L %% 32 == 0 (L = %d)", c->L);
    PGG_CUDA(cudaSetDevice(c->device));
    if (int rc_stage = apply_stage(c)) return rc_stage;
    const size_t bytes = static_cast<size_t>(c->L) * c->L / 8;
    if (c->layout == PGG_BITPACK) {
        PGG_CUDA(cudaMemcpyAsync(host_words_out, c->lat, bytes, cudaMemcpyDeviceToHost, c->stream));
    } else {
        int rc = ensure_staging(c);
        if (rc) return rc;
        PGG_CUDA(pgg::launch_pack(static_cast<const uint8_t *>(c->lat), reinterpret_cast<uint32_t *>(c->staging_d), c->L,
                                  c->stream));
        PGG_CUDA(cudaMemcpyAsync(host_words_out, c->staging_d, bytes, cudaMemcpyDeviceToHost, c->stream));
    }
    PGG_CUDA(cudaStreamSynchronize(c->stream));
    if (step_out) *step_out = c->step;
    return check_status(c);
}

int pgg_set_lattice_packed(pgg_ctx *c, const uint32_t *host_words_in, uint64_t step) {
    g_last_error.clear();
    if (!c || !host_words_in) return fail(PGG_ERR_ARG, "pgg_set_lattice_packed: NULL argument");
    if (c->L % 32 != 0) return fail(PGG_ERR_ARG, "pgg_set_lattice_packed: needs L %% 32 == 0 (L = %d)", c->L);
    if (step >= kMaxStep) return fail(PGG_ERR_ARG, "pgg_set_lattice_packed: step >= 2^56");
    PGG_CUDA(cudaSetDevice(c->device));
    if (int rc_stage = apply_stage(c)) return rc_stage;
    const size_t bytes = static_cast<size_t>(c->L) * c->L / 8;
    if (c->layout == PGG_BITPACK) {
        PGG_CUDA(cudaMemcpyAsync(c->lat, host_words_in, bytes, cudaMemcpyHostToDevice, c->stream));
    } else {
        int rc = ensure_staging(c);
        if (rc) return rc;
        PGG_CUDA(cudaMemcpyAsync(c->staging_d, host_words_in, bytes, cudaMemcpyHostToDevice, c->stream));
        PGG_CUDA(pgg::launch_unpack(reinterpret_cast<const uint32_t *>(c->staging_d), static_cast<uint8_t *>(c->lat), c->L,
                                    c->stream));
    }
    PGG_CUDA(cudaStreamSynchronize(c->stream));
    c->step = step;
    c->running_valid = false;
    c->cls_valid = false;
    return PGG_OK;
}


int pgg_stage_lattice_packed(pgg_ctx *c, const uint32_t *host_words_in, uint64_t step) {
    g_last_error.clear();
    if (!c || !host_words_in) return fail(PGG_ERR_ARG, "pgg_stage_lattice_packed: NULL argument");
    if (c->L % 32 != 0) return fail(PGG_ERR_ARG, "pgg_stage_lattice_packed: needs L %% 32 == 0 (L = %d)", c->L);
    if (step >= kMaxStep) return fail(PGG_ERR_ARG, "pgg_stage_lattice_packed: step >= 2^56");
    if (c->stage_pending >= 0)
        return fail(PGG_ERR_STATE, "pgg_stage_lattice_packed: a staged lattice is still waiting for the call that applies it");
    PGG_CUDA(cudaSetDevice(c->device));
    int rc = ensure_stage(c);
    if (rc) return rc;
    const int b = c->stage_next;
    PGG_CUDA(cudaStreamWaitEvent(c->copy_stream, c->stage_free[b], 0));
    PGG_CUDA(cudaMemcpyAsync(c->stage_d[b], host_words_in, static_cast<size_t>(c->L) * c->L / 8,
                             cudaMemcpyHostToDevice, c->copy_stream));
    PGG_CUDA(cudaEventRecord(c->stage_ready[b], c->copy_stream));
    c->stage_next = b ^ 1;
    c->stage_pending = b;
    c->stage_step = step;
    return PGG_OK;
}

int pgg_get_state(const pgg_ctx *c, uint64_t *seed_out, uint64_t *step_out) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_get_state: NULL context");
    if (seed_out) *seed_out = c->seed;
    if (step_out) *step_out = c->stage_pending >= 0 ? c->stage_step : c->step;
    return PGG_OK;
}

int pgg_set_schedule(pgg_ctx *c, int kernel, int steps_per_launch, int tile_x, int tile_y) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_set_schedule: NULL context");
    if (kernel != PGG_KERNEL_AUTO && kernel != PGG_KERNEL_SIMPLE && kernel != PGG_KERNEL_TILED &&
        kernel != PGG_KERNEL_DIRECT && kernel != PGG_KERNEL_RESIDENT)
        return fail(PGG_ERR_ARG, "pgg_set_schedule: unknown kernel %d", kernel);
    if (kernel == PGG_KERNEL_RESIDENT) {
        const int bands = pgg::resident_bands(c->layout, c->L, c->sms, c->smem_optin);
        if (bands < 1)
            return fail(PGG_ERR_ARG, "pgg_set_schedule: this lattice cannot be resident (L %% 256 == 0, rows within shared memory)");
        if (tile_y != 0 && tile_y != 1 && tile_y != 2 && tile_y != 4)
            return fail(PGG_ERR_ARG, "pgg_set_schedule: resident steps per halo exchange (tile_y) must be 1, 2 or 4");
        const int smax = pgg::resident_max_steps_per_exchange(c->L, bands, c->smem_optin);
        if (tile_y > smax)
            return fail(PGG_ERR_ARG, "pgg_set_schedule: %d steps per halo exchange do not fit (at most %d for L = %d)", tile_y, smax, c->L);
        c->kernel = kernel;
        c->k_fuse = 16;
        c->tile_x = 0;
        c->tile_y = tile_y;
        return PGG_OK;
    }
    if (kernel == PGG_KERNEL_DIRECT) {
        if (!pgg::direct_supported(c->layout, c->L))
            return fail(PGG_ERR_ARG, "pgg_set_schedule: the direct kernel needs a bit-packed lattice with L %% 256 == 0");
        if (tile_x != 0 && tile_x != 4 && tile_x != 8)
            return fail(PGG_ERR_ARG, "pgg_set_schedule: direct kernel words per thread must be 4 or 8");
        if (tile_y != 0 && tile_y != 64 && tile_y != 128 && tile_y != 256)
            return fail(PGG_ERR_ARG, "pgg_set_schedule: direct kernel block size must be 64, 128 or 256");
        c->kernel = kernel;
        c->k_fuse = 1;
        c->tile_x = tile_x;
        c->tile_y = tile_y;
        return PGG_OK;
    }
    if (kernel == PGG_KERNEL_TILED) {
        if (!tiled_supported(c)) return fail(PGG_ERR_ARG, "pgg_set_schedule: the tiled kernel needs L %% 64 == 0 (L = %d)", c->L);
        if (!is_pow2_fuse(steps_per_launch))
            return fail(PGG_ERR_ARG, "pgg_set_schedule: steps_per_launch must be 1, 2, 4, 8 or 16");
        if (tile_x < 0 || tile_x % 64 != 0) return fail(PGG_ERR_ARG, "pgg_set_schedule: tile_x must be a multiple of 64");
        if (tile_y < 0 || tile_y % 4 != 0) return fail(PGG_ERR_ARG, "pgg_set_schedule: tile_y must be a multiple of 4");
        const int tx = tile_x == 0 ? (c->L >= 1024 ? 1024 : c->L) : (tile_x > c->L ? c->L : tile_x);
        const int ty = tile_y == 0 ? 64 : (tile_y > c->L ? c->L : tile_y);
        if (pgg::tiled_smem_bytes(c->layout, c->game, steps_per_launch, tx, ty) == 0)
            return fail(PGG_ERR_ARG, "pgg_set_schedule: tile %dx%d with %d fused steps does not fit in shared memory", tx, ty, steps_per_launch);
    }
    c->kernel = kernel;
    c->k_fuse = kernel == PGG_KERNEL_TILED ? steps_per_launch : 1;
    c->tile_x = kernel == PGG_KERNEL_TILED ? tile_x : 0;
    c->tile_y = kernel == PGG_KERNEL_TILED ? tile_y : 0;
    return PGG_OK;
}

int pgg_set_spin_limit(pgg_ctx *c, unsigned int limit) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_set_spin_limit: NULL context");
    c->spin_limit = limit;
    return PGG_OK;
}

int pgg_set_kernel_timing(pgg_ctx *c, int enable) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_set_kernel_timing: NULL context");
    PGG_CUDA(cudaSetDevice(c->device));
    PGG_CUDA(cudaStreamSynchronize(c->stream));  // no recorded event is still pending
    if (enable) {
        c->tev_used = 0;
    } else {
        timing_release(c);
    }
    c->timing = enable != 0;
    return PGG_OK;
}

int pgg_kernel_time(pgg_ctx *c, double *ms_total, int64_t *launches) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_kernel_time: NULL context");
    PGG_CUDA(cudaSetDevice(c->device));
    PGG_CUDA(cudaStreamSynchronize(c->stream));
    double total = 0.0;
    for (size_t i = 0; i < c->tev_used; ++i) {
        float ms = 0.0f;
        PGG_CUDA(cudaEventElapsedTime(&ms, c->tev_start[i], c->tev_stop[i]));
        total += ms;
    }
    if (ms_total) *ms_total = total;
    if (launches) *launches = static_cast<int64_t>(c->tev_used);
    return PGG_OK;
}

int pgg_get_schedule(const pgg_ctx *c, int *kernel, int *steps_per_launch, int *tile_x, int *tile_y) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_get_schedule: NULL context");
    const Schedule s = resolve_schedule(c);
    if (kernel) *kernel = s.kernel;
    if (steps_per_launch) *steps_per_launch = s.k;
    if (tile_x) *tile_x = s.tile_x;
    if (tile_y) *tile_y = s.tile_y;
    return PGG_OK;
}

int pgg_get_threshold_table(const pgg_ctx *c, uint32_t *host_out) {
    g_last_error.clear();
    if (!c || !host_out) return fail(PGG_ERR_ARG, "pgg_get_threshold_table: NULL argument");
    std::memcpy(host_out, c->table_h, sizeof c->table_h);
    return PGG_OK;
}

int pgg_threshold_table(int game, double r, double K, const double payoff[4], uint32_t *host_out) {
    g_last_error.clear();
    if (!host_out) return fail(PGG_ERR_ARG, "pgg_threshold_table: NULL output");
    if (!(K > 0.0) || !std::isfinite(K)) return fail(PGG_ERR_ARG, "pgg_threshold_table: need K > 0");
    if (game == PGG_GAME_GROUP) {
        if (!(r > 0.0) || !std::isfinite(r)) return fail(PGG_ERR_ARG, "pgg_threshold_table: need r > 0");
        pgg::build_threshold_table(r, K, host_out);
        return PGG_OK;
    }
    if (game != PGG_GAME_PAIRWISE) return fail(PGG_ERR_ARG, "pgg_threshold_table: unknown game %d", game);
    if (!payoff) return fail(PGG_ERR_ARG, "pgg_threshold_table: the pairwise game needs its payoff matrix");
    for (int q = 0; q < 4; ++q)
        if (!std::isfinite(payoff[q])) return fail(PGG_ERR_ARG, "pgg_threshold_table: payoff[%d] is not finite", q);
    pgg::build_pair_threshold_table(payoff, K, host_out);
    return PGG_OK;
}

int pgg_lattice_device_ptr(pgg_ctx *c, void **dev_ptr, uint64_t *bytes) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_lattice_device_ptr: NULL context");
    PGG_CUDA(cudaSetDevice(c->device));
    if (int rc_stage = apply_stage(c)) return rc_stage;
    if (dev_ptr) *dev_ptr = c->lat;
    c->cls_valid = false;  // the caller may write the lattice through the pointer
    if (bytes) *bytes = c->lat_bytes;
    return PGG_OK;
}

int pgg_autotune(pgg_ctx *c, int n_mcs, int *kernel, int *steps_per_launch, int *tile_x, int *tile_y,
                 float *ms_per_mcs) {
    g_last_error.clear();
    if (!c) return fail(PGG_ERR_ARG, "pgg_autotune: NULL context");
    if (n_mcs < 1 || n_mcs > 1000) return fail(PGG_ERR_ARG, "pgg_autotune: n_mcs must be in [1, 1000]");
    PGG_CUDA(cudaSetDevice(c->device));
    if (int rc_stage = apply_stage(c)) return rc_stage;
    // candidates
    std::vector<Schedule> cand;
    if (const int bands = pgg::resident_bands(c->layout, c->L, c->sms, c->smem_optin)) {
        const int smax = pgg::resident_max_steps_per_exchange(c->L, bands, c->smem_optin);
        for (int spe = 1; spe <= smax; spe *= 2) cand.push_back({PGG_KERNEL_RESIDENT, 16, 0, spe});
    }
    if (pgg::direct_supported(c->layout, c->L))
        for (int upt : {4, 8})
            for (int blk : {64, 128, 256}) cand.push_back({PGG_KERNEL_DIRECT, 1, upt, blk});
    if (tiled_supported(c)) {
        const int tiles[][2] = {{2048, 128}, {1024, 256}, {1024, 128}, {1024, 64}, {512, 128}, {512, 64},
                                {256, 64}, {256, 32}, {128, 32}, {128, 16}, {64, 16}, {64, 8}};
        for (int k : {1, 2, 4, 8})
            for (const auto &t : tiles) {
                if (t[0] > c->L || t[1] > c->L) continue;
                if (pgg::tiled_smem_bytes(c->layout, c->game, k, t[0], t[1]) == 0) continue;
                cand.push_back({PGG_KERNEL_TILED, k, t[0], t[1]});
            }
    }
    cand.push_back({PGG_KERNEL_SIMPLE, 1, 0, 0});
    // trials run on the context's own buffers from a saved copy of the state
    void *saved = nullptr;
    cudaError_t e = cudaMalloc(&saved, c->lat_bytes);
    if (e != cudaSuccess) return fail(PGG_ERR_OOM, "pgg_autotune: cudaMalloc(saved lattice): %s", cudaGetErrorString(e));
    const uint64_t step0 = c->step;
    const int kern0 = c->kernel, k0 = c->k_fuse, tx0 = c->tile_x, ty0 = c->tile_y;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Schedule best{PGG_KERNEL_SIMPLE, 1, 0, 0};
    float best_ms = 1e30f;
    int rc = PGG_OK;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
        (e = cudaMemcpyAsync(saved, c->lat, c->lat_bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) {
        rc = fail(PGG_ERR_CUDA, "pgg_autotune: %s", cudaGetErrorString(e));
    }
    for (size_t i = 0; rc == PGG_OK && i < cand.size(); ++i) {
        const Schedule &s = cand[i];
        c->kernel = s.kernel;
        c->k_fuse = s.k;
        c->tile_x = s.tile_x;
        c->tile_y = s.tile_y;
        float ms = 0;
        for (int rep = 0; rep < 2 && rc == PGG_OK; ++rep) {  // rep 0 warms up
            if ((e = cudaMemcpyAsync(c->lat, saved, c->lat_bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) {
                rc = fail(PGG_ERR_CUDA, "pgg_autotune: restore: %s", cudaGetErrorString(e));
                break;
            }
            c->step = step0;
            c->running_valid = false;
            c->cls_valid = false;
            if ((e = cudaEventRecord(e0, c->stream)) != cudaSuccess) { rc = fail(PGG_ERR_CUDA, "pgg_autotune: %s", cudaGetErrorString(e)); break; }
            rc = pgg_step_mcs(c, n_mcs, nullptr);
            if (rc) break;
            if ((e = cudaEventRecord(e1, c->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
                rc = fail(PGG_ERR_CUDA, "pgg_autotune: timing: %s", cudaGetErrorString(e));
        }
        if (rc == PGG_OK && ms / n_mcs < best_ms) {
            best_ms = ms / n_mcs;
            best = s;
        }
    }
    // restore the state and the caller's schedule
    if (saved) {
        cudaMemcpyAsync(c->lat, saved, c->lat_bytes, cudaMemcpyDeviceToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
        cudaFree(saved);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->step = step0;
    c->running_valid = false;
    c->cls_valid = false;
    c->kernel = kern0;
    c->k_fuse = k0;
    c->tile_x = tx0;
    c->tile_y = ty0;
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tuned_mutex);
        g_tuned[std::make_tuple(c->device, c->L, c->layout, c->game)] = best;
    }
    if (kernel) *kernel = best.kernel;
    if (steps_per_launch) *steps_per_launch = best.k;
    if (tile_x) *tile_x = best.tile_x;
    if (tile_y) *tile_y = best.tile_y;
    if (ms_per_mcs) *ms_per_mcs = best_ms;
    return PGG_OK;
}

void pgg_destroy(pgg_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    release_stage(c);
    if (c->lat) cudaFree(c->lat);
    if (c->lat_alt) cudaFree(c->lat_alt);
    if (c->table_d) cudaFree(c->table_d);
    if (c->counts_d) cudaFree(c->counts_d);
    if (c->staging_d) cudaFree(c->staging_d);
    if (c->running_d) cudaFree(c->running_d);
    if (c->mailbox_d) cudaFree(c->mailbox_d);
    if (c->ctr_d) cudaFree(c->ctr_d);
    if (c->count_slots_d) cudaFree(c->count_slots_d);
    if (c->cls_d) cudaFree(c->cls_d);
    if (c->status_d) cudaFree(c->status_d);
    if (c->status_h) cudaFreeHost(c->status_h);
    timing_release(c);
    if (c->counts_h) cudaFreeHost(c->counts_h);
    delete c;
}

}  // extern "C"
