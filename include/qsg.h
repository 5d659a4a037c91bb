/*
 * qsg.h -- C ABI of the GB300 (sm_103a) Monte Carlo library for the
 * Trotter-Suzuki representation of the two-dimensional +-1 Ising spin glass
 * in a transverse field (arXiv 2310.07486, "The Quantum Transition of the
 * Two-Dimensional Ising Spin Glass: A Tale of Two Gaps").
 *
 * Model (Methods, Eq. (Trotter-action) and Eq. (P-S-tau)): classical spins
 * S_{x,tau} = +-1 on an L x L x L_tau lattice, periodic in space, periodic
 * (PBC) or antiperiodic (APBC, only along tau) in imaginary time, with weight
 * exp(-k E(S)) and action
 *     E(S) = - sum_tau [ sum_<x,y> J_xy S_x,tau S_y,tau + sum_x S_x,tau S_x,tau+1 ].
 * Space bonds carry k J_xy and time bonds k; the transverse field of Eq. (H-def)
 * is Gamma = -ln(tanh k) / (2k).  Couplings J_xy = +-1 with probability 1/2
 * (Methods, "Model and simulations").
 *
 * Storage (multispin coding): spins of 64 disorder samples share one uint64
 * word; bit b of word w is sample 64 w + b and a set bit means S = -1.  A
 * "slot" is one lattice of L*L*L_tau words for the word-group w, replica r and
 * ladder position j, slot = (w * R + r) * K + j, words ordered [tau][y][x].
 * Parallel tempering moves spin bits between the slots of one (w, r), so the
 * lattice in slot (w, r, j) is always simulated at k_j.
 *
 * Randomness: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed
 * (low word first).  Counters, with gid the group index:
 *   couplings   (n = y L + x, dir, w, 1<<24 | gid<<8): bits of out[0] | out[1]<<32
 *   hot start   (n, 0, slot, 2<<24 | gid<<8):           bits of out[0] | out[1]<<32
 *   sweep       (block, sweep, slot, 3<<24 | gid<<8): rows are cut into column
 *               pairs starting at x = y & 1 (odd rows pair (1,2), ..., (L-1,0));
 *               with xs = (x - (y & 1)) mod L, site (x, y, tau) takes
 *               out[(tau & 1) * 2 + (xs & 1)], block = ((tau/2) L + y)(L/2) + xs/2;
 *               one 32-bit uniform per site, sweep and slot, shared by the 64
 *               samples of the word
 *   tempering   (16 i + b/4, swap index, w R + r, 4<<24 | gid<<8): sample bit b
 *               of pair i takes out[b & 3]
 *
 * Acceptance is an integer comparison u < T against 32-bit tables built on the
 * host in FP64 (Methods, "Simulation details"):
 *   Metropolis  flip iff S h <= 0 or u < floor(2^32 exp(-(2 k (S h))))
 *   heat bath   S = +1 iff u < min(floor(2^32 / (1 + exp(-(2 k h)))), 2^32 - 1)
 *   tempering   pairs i = 0 .. K-2 in order; swap iff E_{i+1} >= E_i or
 *               u < (A_i[n >> 6] * B_i[n & 63]) >> 32, n = E_i - E_{i+1},
 *               A_i[m] = floor(2^32 exp(-(d_i (64 m)))), B_i[r] = floor(2^32 exp(-(d_i r))),
 *               d_i = k_{i+1} - k_i (uint64 product)
 * where h = sum_space J S_nb + sum_time s S_nb (s = -1 on the APBC wrap bond).
 *
 * Conventions: every call returns a qsg_status and nothing is thrown across
 * the ABI.  Device work is enqueued on the caller's CUDA stream; calls named
 * read_* / get_* / set_* synchronise that stream (except
 * qsg_read_correlators_async and the *_device calls), no other call does
 * (qsg_wait_correlators waits for the asynchronous copies only).  The
 * library allocates no device memory: the caller passes one device workspace
 * of qsg_workspace_bytes() bytes, owned by the caller and used by the library
 * until qsg_destroy().  Host pointers passed to a call are read or written
 * only during that call.
 */
#ifndef QSG_H
#define QSG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qsg_ctx qsg_ctx;

typedef enum {
    QSG_OK = 0,
    QSG_ERR_ARG = -1,       /* null pointer, bad group index, bad ladder, bad count */
    QSG_ERR_SHAPE = -2,     /* L or L_tau odd or out of range, counts < 1 */
    QSG_ERR_CUDA = -3,      /* a CUDA runtime call failed (see qsg_last_cuda_error) */
    QSG_ERR_TIMEOUT = -4,   /* a bounded device wait gave up; results are invalid */
    QSG_ERR_STATE = -5,     /* call out of order (e.g. sweep before init) */
    QSG_ERR_WORKSPACE = -6  /* workspace missing, misaligned or too small */
} qsg_status;

enum { QSG_METROPOLIS = 0, QSG_HEATBATH = 1 };
enum { QSG_PBC = 0, QSG_APBC = 1 };

/* One group of disorder samples that share (L, L_tau, R, K, algorithm,
 * boundary).  Several groups of different sizes may live in one context. */
typedef struct {
    int32_t L;          /* linear size, even, 2 <= L <= 32 */
    int32_t Ltau;       /* Trotter slices, even, 2 <= L_tau <= 65536 */
    int32_t n_samples;  /* disorder samples, >= 1 (stored in ceil(n/64) words) */
    int32_t n_replicas; /* independent replicas per sample and k, 1 <= R <= 1023 */
    int32_t n_k;        /* ladder length K, 1 <= K <= 128 */
    int32_t algo;       /* QSG_METROPOLIS or QSG_HEATBATH */
    int32_t boundary;   /* QSG_PBC or QSG_APBC (along tau only; Methods, Trotter-Suzuki) */
    int32_t reserved;   /* must be 0 */
} qsg_shape;

/* Bytes of device workspace needed for these groups (0 on invalid shapes). */
size_t qsg_workspace_bytes(const qsg_shape *shapes, int32_t n_groups);

/* Create a context over a caller-owned device workspace (256-byte aligned,
 * at least qsg_workspace_bytes() bytes) on CUDA stream `cuda_stream`
 * (a cudaStream_t, may be NULL for the legacy default stream). */
qsg_status qsg_create(qsg_ctx **out, const qsg_shape *shapes, int32_t n_groups, void *d_workspace,
                      size_t workspace_bytes, void *cuda_stream);
void qsg_destroy(qsg_ctx *ctx);
qsg_status qsg_set_stream(qsg_ctx *ctx, void *cuda_stream);

/* Draw the couplings J of every sample (Methods, "Model and simulations"),
 * the hot-start configurations of every slot, build the acceptance tables
 * from the k ladders and clear all accumulators and counters.
 * k_ladders (host): for each group in order, n_k values 0 < k_0 < ... < k_{K-1} < 3. */
qsg_status qsg_init_samples(qsg_ctx *ctx, uint64_t seed, const double *k_ladders);

/* Replace the couplings of one group (host int8 [n_samples][2][L][L] of +-1;
 * [.][0][y][x] couples (x,y)-(x+1,y), [.][1][y][x] couples (x,y)-(x,y+1)).
 * Clears the cached actions.  Synchronises the stream. */
qsg_status qsg_set_couplings(qsg_ctx *ctx, int32_t group, const int8_t *J_host);

/* n_sweeps full checkerboard sweeps of every slot of every group (Methods,
 * "Simulation details"; colour (x+y+tau) mod 2, colour 0 then colour 1).
 * Advances the sweep counter by n_sweeps. */
qsg_status qsg_sweep(qsg_ctx *ctx, int32_t n_sweeps);

/* One parallel-tempering step over the k ladder of every (sample, replica)
 * (Methods, "Simulation details"), using the action of the current
 * configurations.  Accepted swaps exchange the spin bits of that sample between
 * the two slots.  Advances the swap counter. */
qsg_status qsg_tempering_swap(qsg_ctx *ctx);

/* Accumulate, in int64 on the device, for every slot and sample bit
 *   C_acc[r][b][j][tau] += sum_tau1 s c(tau1, tau),  Q_acc[r][b][j][tau] += sum_tau1 c(tau1, tau)^2,
 * c = sum_x S_x,tau1 S_x,tau1+tau (s = -1 when tau1+tau wraps under APBC), and
 *   P_acc[b][j] += sum_{r<r'} sum_tau1 (sum_x S^r_x,tau1 S^r'_x,tau1)^2
 * for tau = 0 .. L_tau/2 (Eqs. (C_A_transfer), (def-C-Q2-tau); the replica
 * overlap is the Tr M^2 / L^2D comparator of the Q2 plateau).
 * The same pass accumulates the one-time sums (Methods, "One-time
 * observables", Eqs. (def-M), (chi-r), (Binder)) over slices tau and replica
 * pairs / triples, with Q_ab = sum_x S^a_x S^b_x and n_c the overlap summed
 * over column (row) c of the slice:
 *   P4[b][j]   += Q_ab^4                                   (128-bit exact)
 *   G[b][j][d] += sum_c n_c (n_{c+d} + n_{c-d})  both directions, d = 0 .. L/2
 *                 (a single term at d = 0 and d = L/2)
 *   T3[b][j]   += Q_ab Q_bc Q_ca                            (3 <= R <= 8)
 *   F3[b][j][d] += Q_uv sum_c n^su_c (n^sv_{c+d} + n^sv_{c-d}), s = a, b, c
 * unless QSG_OPT_ONETIME = 1 turned the three-replica sums off. */
qsg_status qsg_measure_correlators(qsg_ctx *ctx);

/* FP64 finish of one group on the device (Eq. (def-C-Q2-tau)):
 *   C = C_acc / (n_meas L^2 L_tau), Q2 = Q_acc / (n_meas L^4 L_tau),
 *   q2 = P_acc / (n_meas n_pairs L^4 L_tau), n_pairs = R (R-1) / 2,
 * then copied to host buffers C, Q2 [R][n_samples][K][L_tau/2+1] and
 * q2 [n_samples][K] (any may be NULL).  raw (optional, host int64) receives
 * C_acc then Q_acc then P_acc in the same layouts.  Synchronises the stream. */
qsg_status qsg_read_correlators(qsg_ctx *ctx, int32_t group, double *C, double *Q2, double *q2, int64_t *raw);

/* qsg_read_correlators without the host wait: the finish and the copies
 * (same outputs and layouts) run on copy_stream (a cudaStream_t other than
 * the context's) once the work queued so far on the context's stream is done,
 * so the context's stream goes on without them.  The
 * call returns once the work is queued; the host buffers (page-locked for the
 * copies to overlap compute) hold the results once qsg_wait_correlators
 * returns or copy_stream has been synchronised, and must stay allocated until
 * then.  Every later call of the context that writes the correlator buffers
 * (qsg_measure_correlators, a read, qsg_init_samples) is ordered after the
 * copies on the device, so the caller may go on measuring at once.  The
 * device flag is copied with the results and reported by
 * qsg_wait_correlators.  QSG_ERR_ARG for a NULL or the context's own stream. */
qsg_status qsg_read_correlators_async(qsg_ctx *ctx, int32_t group, double *C, double *Q2, double *q2, int64_t *raw,
                                      void *copy_stream);

/* Blocks until the copies of the last qsg_read_correlators_async are done.
 * QSG_ERR_TIMEOUT if the device flag was set by then (as qsg_read_correlators
 * reports it), QSG_OK otherwise or when no asynchronous read is pending. */
qsg_status qsg_wait_correlators(qsg_ctx *ctx);

/* One-time observables of one group (Methods, "One-time observables";
 * Eqs. (chi-r), (xi-r), (Binder)) and the linear susceptibility (Sect. "On the
 * magnetic susceptibilities"), finished in FP64 on the device from the sums
 * of qsg_measure_correlators (N = L^2 sites, p = 2 pi / L along x and y):
 *   per_sample [n_samples][K][7]: q2 = <Q^2>/N^2, q4 = <Q^4>/N^4,
 *     chi2 = <Q^2>/N, F2 = <|Q(p)|^2>/N, chi3 = <Q_ab Q_bc Q_ca>/N,
 *     F3 = <Re Q_su(p) Q_sv(-p) Q_uv>/N, chi_lin = C(0) + 2 sum_{0<tau<L_tau/2}
 *     C(tau) + C(L_tau/2) (C averaged over replicas), where <.> averages
 *     measurements, slices and replica pairs (triples; both p and the three
 *     choices of s for F); chi3 and F3 are NaN unless 3 <= R <= 8 and the
 *     three-replica sums are on;
 *   per_k [K][8]: disorder averages over the group's samples of chi2, F2, then
 *     xi2 = sqrt(chi2/F2 - 1) / (2 sin(pi/L)), chi3, F3, xi3 likewise,
 *     B = mean q4 / (mean q2)^2, and chi_lin;
 *   raw (host int64) [n_samples][K][4 + 2 (L/2+1)]: sum Q^2, sum Q^4 as low
 *     then high 64 bits of a 128-bit integer, T3, G[0..L/2], F3[0..L/2].
 * Any output may be NULL.  Synchronises the stream. */
qsg_status qsg_read_onetime(qsg_ctx *ctx, int32_t group, double *per_sample, double *per_k, int64_t *raw);

/* Per-sample correlation lengths (Methods, "Fitting process and Euclidean
 * correlation length estimation"), host FP64, no device work.
 * C, Q2: host [n_replicas][n_series][L_tau/2+1], e.g. the outputs of
 * qsg_read_correlators with n_series = n_samples * K.  For every series:
 * replica mean and standard error; Q2 plateau = weighted constant on
 * [L_tau/4, L_tau/2] (acceptable iff chi2/dof <= 2); windows tau_w = first lag
 * >= 1 where C (resp. Q2 - plateau) <= 3.5 sigma (Q2: L_tau/2 and the plateau
 * free when the constant fit is not acceptable; C: eta not estimated when C
 * never gets there); C fitted to B [e^{-tau/eta} + z e^{-(L_tau-tau)/eta}]
 * (z = +1 PBC, -1 APBC) on [tau_min, tau_w], tau_min from tau_w/10 up until
 * chi2/dof < 1; Q2 fitted to the plateau plus one and plus two exponentials,
 * tau_min from 1 up until chi2/dof < 0.5, the smaller chi2/dof kept and eta_e
 * its largest decay length.  Diagonal covariance; errors from (J^T W J)^-1.
 * n_replicas >= 2, L_tau >= 4 even.  out: caller-owned [n_series]. */
typedef struct {
    int32_t C_ok, C_tau_w, C_tau_min, Q_ok;
    int32_t Q_tau_w, Q_tau_min, Q_n_exp, plateau_ok;
    double eta, eta_err, C_amp, C_chi2dof;
    double Q_pl, Q_pl_err, plateau_chi2dof, eta_e, eta_e_err, eta_2, Q_chi2dof;
} qsg_fit_result;
qsg_status qsg_fit_correlators(const double *C, const double *Q2, int32_t n_replicas, int64_t n_series,
                               int32_t Ltau, int32_t boundary, qsg_fit_result *out);

/* tilde tau = (L_tau / pi) sin(pi tau / L_tau) for tau = 0 .. L_tau/2 (Sect. "On
 * the magnetic susceptibilities"), into host out[L_tau/2+1]. */
void qsg_tau_tilde(int32_t Ltau, double *out);

/* Sum over measurements and slices of Q_ab^2 = (sum_x S^a_x S^b_x)^2 for every
 * replica pair a < b, pairs ordered (0,1), (0,2), ..., (R-2,R-1): host int64
 * [n_samples][K][R(R-1)/2] (the per-pair form of the q2 accumulator, used by
 * the thermalisation judge).  Synchronises the stream. */
qsg_status qsg_read_pair_overlaps(qsg_ctx *ctx, int32_t group, int64_t *out);

/* ---------------------------------------------------------------------------
 * Learned k ladder.  The paper has no learned component; these entry points
 * predict a sample's k-ladder spacing and sweep budget from its couplings,
 * with the plain uniform ladder as fallback and the log-binning judge below
 * deciding thermalisation, so the physics results do not depend on them.
 * ------------------------------------------------------------------------- */

/* The 64 coupling features of every sample of one group, host float
 * [n_samples][64], computed on the device from the coupling bit-planes.  A
 * plaquette (x,y) with corners (x,y), (x+1,y), (x,y+1), (x+1,y+1) is frustrated
 * when an odd number of its four bonds is negative.  Each feature is a count
 * over its number of cases, divided in FP64 and rounded once to FP32:
 *   0      frustrated plaquettes
 *   1-5    sites by the sum of their four bonds -4, -2, 0, 2, 4
 *   6-10   sites by the number (0..4) of frustrated plaquettes touching them
 *   11-15  2x2 plaquette blocks at even (x, y) by frustrated count 0..4
 *   16-31  frustrated fraction of each cell (floor(4x/L), floor(4y/L)) of a 4x4
 *          coarse grid, index 16 + 4 cy + cx (0 for empty cells)
 *   32, 33 frustrated pairs at offsets (+1,+1), (+1,-1)
 *   34, 35 negative x bonds, negative y bonds
 *   36-41  plaquette rows by frustrated fraction, bins [i/6, (i+1)/6), last closed
 *   42-47  plaquette columns likewise
 *   48-55  frustrated pairs at offsets (d, 0), d = 1..8 (mod L)
 *   56-63  frustrated pairs at offsets (0, d)
 * Uses the correlator scratch of the context.  Synchronises the stream. */
qsg_status qsg_sample_features(qsg_ctx *ctx, int32_t group, float *out);

/* The predictor: a 64 -> 128 -> 128 -> 33 ReLU MLP, FP32 parameters in the
 * order W1[128][64], b1[128], W2[128][128], b2[128], W3[33][128], b3[33]
 * (qsg_mlp_param_count() = 29089).  Outputs: y[0..31] -> softmax -> fractions
 * f_i of the ladder, k_j = k_min + (k_max - k_min) sum_{i<=j} f_i; y[32] =
 * log2(sweep budget) / 16.  Loss of a batch: mean over its samples of the
 * cross-entropy between softmax(y[0:32]) and the targets t[0:32], plus
 * (y[32] - t[32])^2.  Training: Adam (0.9, 0.999, 1e-8), deterministic.
 * Inference in FP32 or BF16 (weights, inputs and hidden activations rounded
 * to bfloat16 nearest-even, FP32 products and sums).
 * The caller allocates the device workspace (qsg_mlp_workspace_bytes) for up
 * to n_data training samples (and prediction inputs) and batches of at most
 * max_batch (<= 4096) samples; the handle never allocates device memory. */
typedef struct qsg_mlp qsg_mlp;
int32_t qsg_mlp_param_count(void);
size_t qsg_mlp_workspace_bytes(int64_t n_data, int32_t max_batch);
qsg_status qsg_mlp_create(qsg_mlp **out, void *d_workspace, size_t workspace_bytes, int64_t n_data,
                          int32_t max_batch, void *cuda_stream);
void qsg_mlp_destroy(qsg_mlp *mlp);
/* Host float [param_count]; set also clears the Adam state.  Both synchronise. */
qsg_status qsg_mlp_set_params(qsg_mlp *mlp, const float *host);
qsg_status qsg_mlp_get_params(qsg_mlp *mlp, float *host);
/* Training set: host float X [n][64] (features), T [n][33] (targets). */
qsg_status qsg_mlp_set_data(qsg_mlp *mlp, const float *X, const float *T, int64_t n);
/* Loss and gradient (host float [param_count], may be NULL) of the batch of
 * training-set rows idx[0..batch), without updating the parameters. */
qsg_status qsg_mlp_grad(qsg_mlp *mlp, const int32_t *idx, int32_t batch, float *loss, float *grad);
/* `steps` Adam steps with learning rate lr, step s on the rows
 * idx[s*batch .. (s+1)*batch); losses (host float [steps], may be NULL)
 * receives each step's batch loss before its update. */
qsg_status qsg_mlp_train(qsg_mlp *mlp, const int32_t *idx, int32_t steps, int32_t batch, float lr, float *losses);
/* Outputs Y (host float [n][33]) for inputs X (host float [n][64]), n <= n_data. */
qsg_status qsg_mlp_predict(qsg_mlp *mlp, const float *X, int64_t n, int32_t bf16, float *Y);

/* Log-binning thermalisation judge (host FP64).  Bins of sweeps
 * [2^m, 2^(m+1)); E_bins [n_bins][n_samples][n_replicas][n_k]: per replica,
 * the bin mean of the energy per site; q_bins [n_bins][n_samples][n_k][pairs]:
 * per replica pair ((0,1), (0,2), ..., (R-2,R-1), as qsg_read_pair_overlaps),
 * the bin mean of q^2.  Each replica's (pair's) values are averaged over the
 * k values.  Energy: mean over replicas with the standard error of their
 * spread; q^2: mean over pairs with the jackknife standard error over
 * replicas.  first_pass[b] (host int32 [n_samples]) = the first bin
 * m >= n_last - 1 such that each of bins m-1 .. m-n_last+1 agrees with bin m
 * within n_sigma combined standard errors for both, or -1.
 * n_replicas >= 3, n_last >= 2, n_sigma > 0. */
qsg_status qsg_judge(const double *E_bins, const double *q_bins, int32_t n_bins, int32_t n_samples,
                     int32_t n_replicas, int32_t n_k, int32_t n_last, double n_sigma, int32_t *first_pass);

/* Action E of every configuration, host int64 [n_samples][R][K] (ladder
 * position j).  Computes it if no sweep fused it.  Synchronises the stream. */
qsg_status qsg_read_energies(qsg_ctx *ctx, int32_t group, int64_t *E_host);

/* Accepted tempering swaps summed over replicas, host int64 [n_samples][K-1]. */
qsg_status qsg_read_accepts(qsg_ctx *ctx, int32_t group, int64_t *acc_host);

/* Spin words of one group, host uint64 [slots][L_tau][L][L] (checkpoint,
 * tests).  set_spins also clears the cached actions.  Both synchronise. */
qsg_status qsg_get_spins(qsg_ctx *ctx, int32_t group, uint64_t *host);
qsg_status qsg_set_spins(qsg_ctx *ctx, int32_t group, const uint64_t *host);

/* The same state to or from a caller-owned DEVICE buffer of the same layout
 * (slots x L_tau x L x L words, on the context's device), copied on the
 * context's stream without waiting: ordered after the work enqueued before
 * and before the work enqueued after.  A caller that stages the next state in
 * device memory while the current one is being swept (an upload on another
 * stream, synchronised with events) hides the host link behind the compute;
 * the copy itself runs at device-memory speed.  set_spins_device also clears
 * the cached actions.  A null buffer is QSG_ERR_ARG. */
qsg_status qsg_get_spins_device(qsg_ctx *ctx, int32_t group, uint64_t *d_out);
qsg_status qsg_set_spins_device(qsg_ctx *ctx, int32_t group, const uint64_t *d_words);

/* Counters: sweeps done, tempering steps done, measurements accumulated.
 * The sweep and swap counters key the Philox streams, so restoring them with
 * the spins (and the couplings, re-drawn by qsg_init_samples from the same
 * seed) resumes a run bit for bit.  n_meas < 0 leaves the measurement count. */
qsg_status qsg_get_counters(qsg_ctx *ctx, uint32_t *sweeps, uint32_t *swaps, int64_t *n_meas);
qsg_status qsg_set_counters(qsg_ctx *ctx, uint32_t sweeps, uint32_t swaps, int64_t n_meas);

/* Tuning options (apply to every group of the context):
 *   QSG_OPT_SWEEP_KERNEL  0 = automatic, 1 = one thread per site and colour
 *                         (two launches per sweep), 2 = fused tau-wavefront
 *                         (one launch per sweep; needs L_tau % 16 == 0)
 *   QSG_OPT_CHUNK         tau planes per wavefront work unit (0 = automatic;
 *                         otherwise a multiple of 16 that divides every L_tau)
 *   QSG_OPT_WAVEFRONT_VARIANT  form of the wavefront kernel, process-wide:
 *                         0 = one work unit per block with L compiled in
 *                         (L = 8, 12, 16, 20, 24; 72 registers, three blocks of 288
 *                         threads per SM at L = 24), four tau planes per
 *                         block barrier; other L use the
 *                         generic kernel;
 *                         1 = the same with two planes per barrier; 3 = with
 *                         four; 2 = the generic kernel (several units per
 *                         block, L at run time, two blocks per SM)
 *   QSG_OPT_CORR_KERNEL   0 = tensor cores (Gram tiles by tcgen05.mma in FP8,
 *                         exact for +-1 spins), 1 = XOR/popcount on the
 *                         integer pipes
 *   QSG_OPT_PERSISTENT    how the groups of a context are swept:
 *                         0 = automatic (mode 3 when the context has several
 *                         groups), 1 = one launch per group and sweep, in
 *                         group order on the context's stream, 2 = one
 *                         persistent launch per sweep serves every group from
 *                         a work queue, largest groups first (needs one
 *                         algorithm, L <= 24, every L_tau % 16 == 0), 3 = each
 *                         group's sweeps on a stream of its own, forked from
 *                         and joined back into the context's stream (inside
 *                         the CUDA graph when QSG_OPT_GRAPH is on), so that
 *                         the groups' launches overlap and small groups fill
 *                         the last waves of large ones
 *   QSG_OPT_GRAPH         0 = off; G in 1..4096 = qsg_sweep replays a CUDA
 *                         graph of G sweeps (captured on first use and again
 *                         after an option change) for each whole batch of G,
 *                         and launches the remainder directly.  The graph
 *                         reads the sweep index from a device counter, so
 *                         its Philox draws equal those of direct launches.
 *                         Needs the wavefront kernel for every group.
 *   QSG_OPT_ONETIME       0 = accumulate every one-time sum (default),
 *                         1 = skip the three-replica sums (chi3, F3 become
 *                         NaN); only before the first measurement
 *   QSG_OPT_TAIL          0 = every slot in chunks of the same length
 *                         (default); T > 0 = the wavefront launch of a group
 *                         sweeps its last min(T, slots) slots in chunks of a
 *                         quarter of the chunk length (when that is a multiple
 *                         of 16), scheduled after all other units, so that
 *                         short units fill the last wave of blocks
 *   QSG_OPT_WAIT_LIMIT    polls of each bounded device wait of the tensor-core
 *                         correlator pipeline before it gives up (default
 *                         2^22, 0..2^30).  A wait that gives up makes every
 *                         role of the kernel run out its loops without
 *                         further work and sets the context's device flag:
 *                         that measurement is not accumulated, and
 *                         qsg_read_correlators returns QSG_ERR_TIMEOUT from
 *                         then on (the flag stays set for the context).  A
 *                         small value is a way to exercise that path; the
 *                         default never gives up on a working GPU.
 *   QSG_OPT_UNITS_PER_BLOCK  work units (slot, tau chunk) per thread block of
 *                         the generic wavefront kernel, which serves the
 *                         lattice sizes without a compiled kernel: 0 =
 *                         automatic (as many as fit 256 threads, at most 16),
 *                         or 1, 2, 4, 8, 16 (rounded down to at most 512
 *                         threads).  A unit's thread owns two site words of
 *                         a row whatever the grouping.
 * Results do not depend on the options (except QSG_OPT_WAIT_LIMIT set too low
 * for the pipeline to make progress): every kernel produces the same bits. */
enum { QSG_OPT_SWEEP_KERNEL = 1, QSG_OPT_CHUNK = 2, QSG_OPT_WAVEFRONT_VARIANT = 3, QSG_OPT_CORR_KERNEL = 4,
       QSG_OPT_PERSISTENT = 5, QSG_OPT_GRAPH = 6, QSG_OPT_ONETIME = 7, QSG_OPT_TAIL = 8, QSG_OPT_WAIT_LIMIT = 9,
       QSG_OPT_UNITS_PER_BLOCK = 10 };
qsg_status qsg_set_option(qsg_ctx *ctx, int32_t option, int64_t value);

/* Sweeps without any device allocation.  (This entry point has no
 * counterpart in the paper: it is a service for callers of this library.)
 *
 * Some callers cannot allocate device memory themselves: a plugin or service
 * whose GPU memory is owned by the host application's allocator or held to a
 * fixed budget, or code that must avoid the device-wide synchronisation that
 * cudaMalloc and cudaFree can cause.  Such a caller passes its own buffers --
 * d_spins [slots][L_tau][L][L] words (read and written), d_Jx and d_Jy
 * [words][L][L] coupling words as described above -- and this function runs
 * n_sweeps full sweeps of the fused wavefront kernel on them, exactly as
 * qsg_sweep does for a context (the same bits for the same seed, group_id and
 * sweep counter first_sweep).  k_ladder (host) holds the n_k values of the
 * ladder; the acceptance table is built from it on each call.
 *
 * The kernel's scratch (its chunk-boundary arrival counters and the
 * acceptance table) lives in two fixed arrays in device memory that every GPU
 * loading this library holds until the process exits: at most 2^20 counters
 * (slots x tau chunks) and 128 ladder positions.  Shapes beyond these limits
 * are rejected with QSG_ERR_WORKSPACE before any pointer is looked at; shapes
 * with L_tau not a multiple of 16 (or otherwise invalid) with QSG_ERR_SHAPE;
 * null buffers, a bad ladder or a cuda_stream that does not belong to the
 * current device with QSG_ERR_ARG.  The library cannot check the sizes of the
 * caller's buffers: they must hold the words given above.
 * The first call on a device (with that device current) looks the arrays up
 * and clears the counters, so it should come before any stream capture on
 * that device; the addresses are cached per device and do not survive
 * cudaDeviceReset.  Every call shares the same arrays, which keep the last
 * call's contents: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The call copies the
 * table to the device and waits for that copy on cuda_stream; the sweeps are
 * enqueued on cuda_stream without waiting.  Nothing is allocated. */
qsg_status qsg_sweep_static_scratch(uint64_t *d_spins, const uint64_t *d_Jx, const uint64_t *d_Jy,
                                    const qsg_shape *shape, int32_t group_id, const double *k_ladder, uint64_t seed,
                                    uint32_t first_sweep, int32_t n_sweeps, void *cuda_stream);

/* Number of kernels this library has launched in this process (all contexts);
 * a diagnostic for benchmarks and for checking that the GPU path ran. */
uint64_t qsg_kernel_launches(void);

const char *qsg_strerror(qsg_status status);
/* Text of the last CUDA error seen by this context (empty if none). */
const char *qsg_last_cuda_error(qsg_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* QSG_H */
