// pgg_noalloc.cu -- pgg_step_mcs_noalloc: the fused tiled step for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: plug-ins of a host application that
// hands out all device memory from its own pool (a cudaMalloc there fails once the pool has
// taken the device, or escapes the application's accounting), and services that must not
// allocate after start-up because cudaMalloc can block on the whole device and take an unbounded
// time. This entry point takes the caller's input and output lattices and runs the same fused
// tiled kernel as pgg_step_mcs, with the kernel's scratch -- the intermediate lattice between
// the two fused launches of each MCS and the adoption threshold table -- in a fixed,
// file-scope device array instead of memory allocated per context.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pgg.h"
#include "pgg_device.cuh"
#include "pgg_internal.h"

namespace {

// Scratch of the allocation-free entry point: an intermediate lattice of up to
// kNoallocLatticeBytes followed by the threshold table. Every GPU that loads the
// library holds this array until the process exits.
constexpr size_t kNoallocLatticeBytes = size_t(4) << 20;  // 4 MiB
constexpr size_t kNoallocTableOffset = kNoallocLatticeBytes;
constexpr size_t kNoallocScratchBytes = kNoallocLatticeBytes + pgg::kTableEntries * sizeof(uint32_t);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_dev[kMaxDevices];  // device address of g_noalloc_scratch, per device

// Two fused launches of 8 sublattice steps per MCS; tile chosen to fit any allowed L.
constexpr int kFuse = 8;

// The threshold table travels to the device as a kernel parameter (5408 bytes, well inside the
// 32 KB parameter space), so a call needs no host staging buffer and no pageable copy.
struct TableParam {
    uint32_t t[pgg::kTableEntries];
};

__global__ void k_noalloc_table(const __grid_constant__ TableParam p, uint32_t *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < pgg::kTableEntries) dst[i] = p.t[i];
}

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return pgg::record_error(code, buf);
}

// Resolve the device address of the scratch array for the current device, once.
int scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PGG_ERR_CUDA, "pgg_step_mcs_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PGG_ERR_ARG, "pgg_step_mcs_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(PGG_ERR_CUDA, "pgg_step_mcs_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_dev[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_dev[dev];
    return PGG_OK;
}

}  // namespace

extern "C" int pgg_step_mcs_noalloc(const void *lattice_in, void *lattice_out, int L, int layout,
                                    double r, double K, uint64_t seed, uint64_t step0,
                                    int64_t n_mcs, uint64_t *coop_per_mcs, void *cuda_stream) {
    pgg::clear_error();
    if (!lattice_in || !lattice_out) return fail(PGG_ERR_ARG, "pgg_step_mcs_noalloc: NULL lattice");
    if (layout != PGG_U8 && layout != PGG_BITPACK)
        return fail(PGG_ERR_ARG, "pgg_step_mcs_noalloc: unknown layout %d", layout);
    if (L < 64 || L % 64 != 0) return fail(PGG_ERR_ARG, "pgg_step_mcs_noalloc: L = %d must be a multiple of 64", L);
    const size_t bytes = layout == PGG_U8 ? size_t(L) * L : size_t(L) * L / 8;
    if (bytes > kNoallocLatticeBytes)
        return fail(PGG_ERR_ARG,
                    "pgg_step_mcs_noalloc: a %s lattice of L = %d needs %zu bytes of scratch, more than the "
                    "fixed %zu (largest L: %d uint8, %d bit-packed)",
                    layout == PGG_U8 ? "uint8" : "bit-packed", L, bytes, kNoallocLatticeBytes, 2048, 4096);
    if (!(r > 0.0) || !(K > 0.0)) return fail(PGG_ERR_ARG, "pgg_step_mcs_noalloc: need r > 0 and K > 0");
    if (n_mcs < 0) return fail(PGG_ERR_ARG, "pgg_step_mcs_noalloc: n_mcs < 0");
    // step0 + 16 n_mcs < 2^56, tested without forming the sum (which could wrap)
    constexpr uint64_t kMaxStep = 1ull << 56;
    if (step0 >= kMaxStep || static_cast<uint64_t>(n_mcs) > (kMaxStep - 1 - step0) / 16)
        return fail(PGG_ERR_ARG, "pgg_step_mcs_noalloc: step counter would pass 2^56");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    uint32_t *table_d = reinterpret_cast<uint32_t *>(scratch + kNoallocTableOffset);
    TableParam tp;
    pgg::build_threshold_table(r, K, tp.t);
    k_noalloc_table<<<(pgg::kTableEntries + 255) / 256, 256, 0, stream>>>(tp, table_d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && coop_per_mcs && n_mcs > 0)
        e = cudaMemsetAsync(coop_per_mcs, 0, size_t(n_mcs) * sizeof(uint64_t), stream);
    if (e != cudaSuccess) return fail(PGG_ERR_CUDA, "pgg_step_mcs_noalloc: %s", cudaGetErrorString(e));
    const int tile_x = L < 1024 ? L : 1024;
    const int tile_y = L < 128 ? L : 128;
    const void *src = lattice_in;
    for (int64_t m = 0; m < n_mcs; ++m) {
        for (int half = 0; half < 16 / kFuse; ++half) {
            pgg::TiledArgs a;
            a.game = pgg::kGroupGame;
            a.status = nullptr;
            a.src = src;
            a.dst = half == 0 ? static_cast<void *>(scratch) : lattice_out;
            a.L = L;
            a.layout = layout;
            a.seed = seed;
            a.k0 = step0 + 16ull * static_cast<uint64_t>(m) + static_cast<uint64_t>(half * kFuse);
            a.steps = kFuse;
            a.tile_x = tile_x;
            a.tile_y = tile_y;
            a.table = table_d;
            a.count_out = (half == 16 / kFuse - 1 && coop_per_mcs)
                              ? reinterpret_cast<unsigned long long *>(coop_per_mcs + m) : nullptr;
            e = pgg::launch_step_tiled(a, stream);
            if (e != cudaSuccess) return fail(PGG_ERR_CUDA, "pgg_step_mcs_noalloc: tiled launch: %s", cudaGetErrorString(e));
            src = a.dst;
        }
    }
    if (n_mcs == 0 && lattice_in != lattice_out) {
        e = cudaMemcpyAsync(lattice_out, lattice_in, bytes, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return fail(PGG_ERR_CUDA, "pgg_step_mcs_noalloc: %s", cudaGetErrorString(e));
    }
    return PGG_OK;
}
