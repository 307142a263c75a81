// pgg_internal.h -- launchers shared between the C ABI (pgg_abi.cu) and the kernel
// translation units. Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace pgg {

enum Layout { kU8 = 0, kPacked = 1 };

// Host-built adoption thresholds of Eq. (3), 2*26*26 entries indexed
// (s_x*26 + S_x)*26 + S_y (defined in pgg_abi.cu).
void build_threshold_table(double r, double K, uint32_t *T);
// The same for the pairwise game of Section VI with payoff matrix pay = {R, S, T, P}:
// 2*5*5 entries indexed (s_x*5 + n_x)*5 + n_y, the rest of the 2*26*26 buffer zero.
void build_pair_threshold_table(const double pay[4], double K, uint32_t *T);

// Set / clear the calling thread's pgg_last_error() message (defined in pgg_abi.cu).
int record_error(int code, const char *message);
void clear_error();

// Bernoulli(p) initial lattice from the init stream; thr = floor(p 2^32) (2^32 for p = 1).
cudaError_t launch_init(int layout, void *lat, int L, uint64_t seed, uint64_t thr,
                        cudaStream_t s);

// One sublattice step k in place with the per-site baseline kernel.
cudaError_t launch_step_simple(int layout, int game, void *lat, int L, uint64_t seed, uint64_t k,
                               const uint32_t *table, cudaStream_t s);

// *out += number of set bits in buf (bytes % 16 == 0, buf 16-byte aligned). A uint8
// lattice holds 0/1 bytes, so this counts cooperators for both layouts.
cudaError_t launch_popcount(const void *buf, size_t bytes, unsigned long long *out,
                            cudaStream_t s);

// uint8 (0 / non-zero) <-> bit-packed conversion of an L x L lattice (L % 32 == 0).
cudaError_t launch_pack(const uint8_t *src, uint32_t *dst, int L, cudaStream_t s);
cudaError_t launch_unpack(const uint32_t *src, uint8_t *dst, int L, cudaStream_t s);

// Map every non-zero byte to 1 (n % 16 == 0, 16-byte aligned).
cudaError_t launch_normalize(uint8_t *buf, size_t n, cudaStream_t s);

// Tiled, temporally blocked step kernel: `steps` sublattice steps k0 .. k0+steps-1.
// src and dst may be equal only when steps == 1. If count_out is not NULL the
// cooperator count of the result is added to *count_out.
struct TiledArgs {
    int game;  // Game (pgg_device.cuh): the halo is read radius x steps
    const void *src;
    void *dst;
    int L;
    int layout;
    uint64_t seed;
    uint64_t k0;
    int steps;
    int tile_x;  // sites, multiple of 64
    int tile_y;  // sites, multiple of 4
    const uint32_t *table;
    unsigned long long *count_out;
    int *status;  // | 4 when an index check fails (checked build); nullable
};
cudaError_t launch_step_tiled(const TiledArgs &a, cudaStream_t s);

// In-place single sublattice step k on a bit-packed lattice with operands read from global
// memory, upt (4 or 8) words per thread, blocks of `block` (64, 128 or 256) threads;
// *running (if not NULL) += the change in the number of cooperators. Needs L % 256 == 0.
bool direct_supported(int layout, int L);
cudaError_t launch_step_direct(int game, uint32_t *lat, int L, uint64_t seed, uint64_t k, const uint32_t *table,
                               unsigned long long *running, int *status, int upt, int block, cudaStream_t s);
// Shared memory (bytes) the tiled kernel needs for a configuration; 0 if unsupported.
size_t tiled_smem_bytes(int layout, int game, int steps, int tile_x, int tile_y);

// Whole bit-packed lattice resident in shared memory for n_mcs MCS (one cooperative launch,
// one row band per CTA, edge rows exchanged through a mailbox every steps_per_exchange steps).
struct ResidentArgs {
    int game;                     // Game (pgg_device.cuh)
    uint32_t *lat;                // bit-packed lattice, or
    uint8_t *lat8 = nullptr;      // a uint8 lattice (then lat is unused): packed as it is staged
    int L;
    int n_bands;
    uint64_t seed, k0;
    int n_mcs;
    const uint32_t *table;
    uint32_t *mailbox;            // resident_mailbox_words(L, n_bands) words
    unsigned int *ctr;            // n_bands counters
    unsigned int ctr_base;        // a launch publishes ctr_base + completed steps: every value an
                                  // earlier launch left is below it, so ctr needs no reset
    bool reset_ctr;               // zero ctr before the launch (first use, or ctr_base wrapped)
    unsigned long long *counts;   // n_mcs counts (nullable), written by the launch: no zeroing needed
    unsigned long long *count_acc = nullptr;  // kResidentCountSlots sums and
    unsigned int *count_tick = nullptr;       // kResidentCountSlots band tallies, all zero before the
                                              // launch; a launch that ends normally leaves them zero
    int *status;                  // | 1 a bounded wait ran out, | 2 the alignment check failed, | 4 an index
                                  // check failed (checked build), | 8 a CTA stopped with a halo load
                                  // possibly in flight (fatal for the device context)
    unsigned int spin_limit;      // polls before a wait gives up
    int steps_per_exchange = 1;   // sublattice steps between halo exchanges: 1, 2 or 4
    bool class_copy = false;      // keep and scan a column-class copy (resident_class_copy must hold)
    uint32_t *cls_g = nullptr;    // L*L/32 words for the class copy between launches (nullable: rebuilt each launch)
    bool cls_load = false;        // cls_g holds the class copy of this lattice: stage it instead of building it
    unsigned int *hint = nullptr; // n_bands words kept between launches (pass-choice hint), nullable
    unsigned int dense_per_mille = 100;  // a step takes the dense pass when the previous one flipped
                                         // more than this share (per mille) of its sites
};
// Count slots of the resident kernel: MCS m of a launch sums its band counts in slot m mod this.
constexpr int kResidentCountSlots = 64;
int resident_bands(int layout, int L, int sms, size_t smem_optin);
// Largest steps_per_exchange (4, 2 or 1) whose halo rows fit the shared memory.
int resident_max_steps_per_exchange(int L, int n_bands, size_t smem_optin);
size_t resident_mailbox_words(int L, int n_bands);
// Whether the column-class copy fits beside the rows for s steps per exchange.
bool resident_class_copy(int L, int n_bands, int s, size_t smem_optin);
cudaError_t launch_resident(const ResidentArgs &a, cudaStream_t s);

}  // namespace pgg
