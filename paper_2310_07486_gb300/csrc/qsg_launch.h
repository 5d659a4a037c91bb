// qsg_launch.h -- host-side launchers of the sm_103a kernels (internal).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "qsg_device.cuh"

namespace qsg {

// Process-wide count of kernel launches (qsg_kernel_launches()).
void count_launches(int n);

// Acceptance tables of a ladder k[0..K) (host FP64, integer results), 16 words
// per ladder position: [0..2] Metropolis thresholds for S h = 2, 4, 6, [8..14]
// heat-bath thresholds for h = 6 - 2 n, the rest zero.  False if the ladder is
// not 0 < k_0 < ... < k_{K-1} < 3 or a table is not monotone (the bitsliced
// comparison of the sweep kernels relies on monotone tables).
bool build_accept_tables(const double *k, int K, uint32_t *table);

// Device-side status word: non-zero after a bounded wait gave up.
enum : int { DEVERR_NONE = 0, DEVERR_TIMEOUT = 1 };

cudaError_t launch_init_couplings(const Group &g, uint64_t seed, cudaStream_t st);
cudaError_t launch_init_spins(const Group &g, uint64_t seed, cudaStream_t st);

// One full sweep (colour 0 then colour 1) of every slot of the group.
// The "reference" variant runs one launch per colour with one thread per site.
cudaError_t launch_sweep_reference(const Group &g, uint32_t sweep, uint64_t seed, cudaStream_t st);

// The fused wavefront sweep: C = planes per work unit (0 if the group cannot
// use this kernel), arrivals = nslots * (L_tau / 4) zeroed counters.
int wavefront_chunk(const Group &g, int requested);
// 0: one unit per block where k_sweep_unit exists (four planes per
// barrier); 1: two planes per barrier; 3: four (as 0); 2: the generic kernel
extern int g_wavefront_variant;
// The sweep index is *sweep_base + sweep (sweep_base may be null), so that a
// captured CUDA graph of several sweeps can be replayed later.  The last
// `tail` slots (0 = none) run chunks of C / 4 planes after every other unit.
cudaError_t launch_sweep_wavefront(const Group &g, const uint32_t *sweep_base, uint32_t sweep, uint64_t seed,
                                   unsigned *arrivals, int C, int tail, cudaStream_t st);
// The one-unit-per-block form (k_sweep_unit.cu) for L = 20, 24: slots
// [0, S1) in chunks of C planes, the others in chunks of C2; 2 or 4 planes
// per block barrier.
bool sweep_unit_supported(const Group &g);
cudaError_t launch_sweep_unit(const Group &g, int planes_per_barrier, int C, int C2, int S1,
                              const uint32_t *sweep_base, uint32_t sweep, uint64_t seed, unsigned *arrivals,
                              cudaStream_t st);
cudaError_t launch_set_word(uint32_t *p, uint32_t value, cudaStream_t st);
// dst[0..words) = src[0..words), device to device, by a kernel when both are
// 16-byte aligned and words is even (else by cudaMemcpyAsync).
cudaError_t launch_copy_words(uint64_t *dst, const uint64_t *src, size_t words, cudaStream_t st);
cudaError_t launch_add_word(uint32_t *p, uint32_t value, cudaStream_t st);

// All groups of a context in one persistent launch per sweep (same algorithm,
// L <= 24, L_tau % 16 == 0).  Device arrays: the Group structs, the group
// order (largest first), the prefix sums of work units in that order, the
// chunk length of every group, and two queue counters (zero between launches).
struct PersistentPlan {
    const Group *groups;
    const int *order, *prefix, *chunk;
    unsigned *queue;
    int ngroups, total_units, algo;
};
cudaError_t launch_sweep_persistent(const PersistentPlan &plan, const uint32_t *sweep_base, uint32_t sweep,
                                    uint64_t seed, cudaStream_t st);

// Unsatisfied-bond counts U[slot][bit] of the current configurations.
cudaError_t launch_energy(const Group &g, cudaStream_t st);

// Tempering step `m`: decisions (and U bookkeeping), then the spin-bit moves.
cudaError_t launch_tempering(const Group &g, uint32_t m, uint64_t seed, cudaStream_t st);

// Correlator accumulation through the x-packed transposed scratch buffer;
// tensor = 1 computes the Gram tiles with tcgen05 (k_corr_tc.cu), 0 with
// XOR/popcount on the integer pipes.  status receives DEVERR_TIMEOUT if a
// bounded wait of the tensor path gave up (after wait_limit polls).
// triples = 1 also accumulates the three-replica one-time sums (3 <= R <= 8).
constexpr unsigned kDefaultWaitLimit = 1u << 22;
cudaError_t launch_measure(const Group &g, uint64_t *scratch, size_t scratch_words, int tensor, int triples,
                           int *status, unsigned wait_limit, cudaStream_t st);
// One-time observable sums of a batch of (w, j) pairs from the transposed scratch.
cudaError_t launch_onetime(const Group &g, int p0, int np, const uint64_t *P, int triples, cudaStream_t st);
// FP64 finish of the one-time observables into g.outO and g.outK.
cudaError_t launch_onetime_finish(const Group &g, long long n_meas, int triples, cudaStream_t st);
// Tensor-core Gram path over the transposed bits P of a batch: folds every
// 128 x 128 tile of the Gram matrices into the lag sums.
cudaError_t launch_gram_tc(const Group &g, int p0, int npairs, const uint64_t *P, int *status, unsigned wait_limit,
                           cudaStream_t st);
bool gram_tc_fits(const Group &g);  // the tensor-core path's shared memory fits one CTA

// FP64 finish into g.outC / g.outQ / g.outP.
cudaError_t launch_finish(const Group &g, long long n_meas, cudaStream_t st);

// Scratch words the correlator path needs for one (w, j) pair of the group.
size_t measure_scratch_words_per_pair(const Group &g);

// The 64 coupling features of every sample bit of the group, out [W*64][64].
cudaError_t launch_features(const Group &g, float *out, cudaStream_t st);

// Learned-ladder MLP (k_mlp.cu).  P: FP32 parameters, M, V: Adam moments;
// one step = gradient of the batch idx[0..batch) (tiles of 16 samples into
// `partial`), then Adam at step number t if adam != 0; grad_out and loss_out
// (device) may be null.
int mlp_param_count();
cudaError_t launch_mlp_step(float *P, float *M, float *V, const float *X, const float *T, const int *idx, int batch,
                            float *partial, float *loss_partial, float *grad_out, int adam, float lr, int t,
                            float *loss_out, cudaStream_t st);
cudaError_t launch_mlp_infer(const float *P, __nv_bfloat16 *Pb, const float *X, float *Y, long long n, int bf16,
                             cudaStream_t st);

}  // namespace qsg
