"""GPU path (through the C ABI) against the CPU oracle, bit for bit.

Spins, integer actions, tempering decisions and int64 correlator sums must be
identical; the FP64 correlators must agree to 1e-12 relative (they are one
IEEE division of identical integers, so in practice they are identical).
Small cases cover several tiles, ragged sample counts (not a multiple of 64)
and both boundary conditions; the full-size cases run in the bench's launch
configuration and compare one sample, chosen at random, that the oracle
simulates alone.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2310_07486_gb300 import qsg as Q  # noqa: E402
from paper_2310_07486_gb300 import workloads  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _pair(shape, ladder, seed, first=0, n_oracle=None, gid=0):
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(seed, [ladder])
    orc = oracle.OracleGroup(shape.L, shape.Ltau, n_oracle or shape.n_samples, shape.n_replicas, shape.n_k,
                             algo=shape.algo, boundary=shape.boundary, group_id=gid, first_sample=first)
    orc.init(seed, ladder)
    return ctx, orc


def _gpu_spins(ctx, shape, group=0, first=0, n=None):
    words = ctx.qsg_get_spins(group)
    S = Q.unpack_spins(words, shape)
    n = n or shape.n_samples
    return S[first:first + n]


def _check_corr(gpu, orc_res):
    for key in ("C_raw", "Q2_raw", "q2_raw"):
        assert np.array_equal(gpu[key], orc_res[key]), key
    for key in ("C", "Q2", "q2"):
        a, b = gpu[key], orc_res[key]
        both_nan = np.isnan(a) & np.isnan(b)
        assert np.all(both_nan | (np.abs(a - b) <= RTOL * np.maximum(np.abs(b), 1e-300))), key


@pytest.mark.parametrize("algo", [Q.METROPOLIS, Q.HEATBATH])
@pytest.mark.parametrize("boundary", [Q.PBC, Q.APBC])
def test_init_and_sweeps_match_oracle(algo, boundary):
    shape = Q.Shape(8, 12, 70, 2, 2, algo, boundary)  # 2 words, ragged last word
    lad = np.array([0.25, 0.31])
    ctx, orc = _pair(shape, lad, seed=11)
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    assert np.array_equal(ctx.qsg_read_energies(), orc.energies())
    for n in (1, 4):
        ctx.qsg_sweep(n)
        orc.sweep(n)
        assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
        assert np.array_equal(ctx.qsg_read_energies(), orc.energies())


@pytest.mark.parametrize("L,Ltau", [(2, 2), (2, 6), (6, 4), (32, 4)])
def test_edge_shapes_match_oracle(L, Ltau):
    shape = Q.Shape(L, Ltau, 65, 1, 2, Q.METROPOLIS, Q.APBC)
    ctx, orc = _pair(shape, np.array([0.2, 0.4]), seed=5)
    for _ in range(3):
        ctx.qsg_sweep(2)
        orc.sweep(2)
        ctx.qsg_tempering_swap()
        orc.swap()
        ctx.qsg_measure_correlators()
        orc.measure()
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    _check_corr(ctx.qsg_read_correlators(raw=True), orc.read())


@pytest.mark.parametrize("algo", [Q.METROPOLIS, Q.HEATBATH])
def test_tempering_matches_oracle(algo):
    shape = Q.Shape(6, 8, 70, 2, 5, algo, Q.PBC)
    lad = workloads.uniform_ladder(0.15, 0.45, 5)
    ctx, orc = _pair(shape, lad, seed=21)
    for _ in range(8):
        ctx.qsg_sweep(3)
        orc.sweep(3)
        ctx.qsg_tempering_swap()
        orc.swap()
        assert np.array_equal(ctx.qsg_read_energies(), orc.energies())
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    assert np.array_equal(ctx.qsg_read_accepts(), orc.accepts())
    assert ctx.qsg_read_accepts().sum() > 0


def test_tempering_chains_over_a_long_ladder_match_oracle():
    """A dense ladder accepts most swaps, so a configuration often moves
    several positions in one tempering step: the moves walk runs of
    consecutive swapped pairs, and pairs without a swap are skipped."""
    shape = Q.Shape(4, 8, 70, 2, 24, Q.HEATBATH, Q.APBC)
    lad = workloads.uniform_ladder(0.30, 0.33, 24)
    ctx, orc = _pair(shape, lad, seed=5)
    for _ in range(6):
        ctx.qsg_sweep(1)
        orc.sweep(1)
        ctx.qsg_tempering_swap()
        orc.swap()
        assert np.array_equal(ctx.qsg_read_energies(), orc.energies())
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    assert np.array_equal(ctx.qsg_read_accepts(), orc.accepts())
    acc = ctx.qsg_read_accepts()
    assert acc.sum() > 6 * 23 * 70 * 2 // 4  # most pairs swap


@pytest.mark.parametrize("L,Ltau,boundary", [(8, 1026, Q.APBC), (12, 126, Q.PBC), (16, 1024, Q.APBC),
                                             (20, 126, Q.APBC), (24, 1026, Q.PBC), (24, 130, Q.APBC),
                                             (10, 70, Q.PBC)])
def test_energies_of_every_compiled_lattice_size_match_oracle(L, Ltau, boundary):
    # the energy pass has a kernel with L compiled in for L = 8, 12, 16, 20,
    # 24 (runs of 256 planes from L_tau = 1024, else 128; L_tau = 2 mod 4
    # leaves a two-plane step) and a generic one for the other sizes
    shape = Q.Shape(L, Ltau, 1, 2, 3, Q.METROPOLIS, boundary)
    lad = workloads.uniform_ladder(0.25, 0.35, 3)
    ctx, orc = _pair(shape, lad, seed=L + Ltau)
    for _ in range(3):
        ctx.qsg_sweep(1)
        orc.sweep(1)
        ctx.qsg_tempering_swap()
        orc.swap()
        assert np.array_equal(ctx.qsg_read_energies(), orc.energies())
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())


@pytest.mark.parametrize("Ltau,boundary", [(70, Q.APBC), (130, Q.PBC), (130, Q.APBC)])
def test_energies_with_ragged_plane_runs_match_oracle(Ltau, boundary):
    # the energy pass takes 128-plane runs, four planes per step: L_tau = 70
    # ends a run two planes into a step, L_tau = 130 leaves a second run of two
    shape = Q.Shape(8, Ltau, 70, 2, 3, Q.HEATBATH, boundary)
    lad = workloads.uniform_ladder(0.2, 0.4, 3)
    ctx, orc = _pair(shape, lad, seed=33)
    for _ in range(4):
        ctx.qsg_sweep(2)
        orc.sweep(2)
        ctx.qsg_tempering_swap()
        orc.swap()
        assert np.array_equal(ctx.qsg_read_energies(), orc.energies())
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    assert np.array_equal(ctx.qsg_read_accepts(), orc.accepts())


@pytest.mark.parametrize("boundary", [Q.PBC, Q.APBC])
def test_correlators_match_oracle(boundary):
    shape = Q.Shape(10, 40, 66, 3, 2, Q.HEATBATH, boundary)  # L^2 = 100: two x-packed words, ragged
    lad = np.array([0.28, 0.33])
    ctx, orc = _pair(shape, lad, seed=8)
    for _ in range(4):
        ctx.qsg_sweep(2)
        orc.sweep(2)
        ctx.qsg_measure_correlators()
        orc.measure()
    gpu = ctx.qsg_read_correlators(raw=True)
    _check_corr(gpu, orc.read())
    assert np.all(gpu["C"][..., 0] == 1.0) and np.all(gpu["Q2"][..., 0] == 1.0)


def test_two_groups_of_different_size():
    shapes = [Q.Shape(6, 8, 3, 2, 3, Q.METROPOLIS, Q.PBC), Q.Shape(8, 16, 66, 2, 2, Q.HEATBATH, Q.APBC)]
    lads = [np.array([0.2, 0.3, 0.4]), np.array([0.25, 0.35])]
    ctx = Q.Context(shapes)
    ctx.qsg_init_samples(17, lads)
    orcs = []
    for gid, (s, l) in enumerate(zip(shapes, lads)):
        o = oracle.OracleGroup(s.L, s.Ltau, s.n_samples, s.n_replicas, s.n_k, algo=s.algo, boundary=s.boundary,
                               group_id=gid)
        o.init(17, l)
        orcs.append(o)
    for _ in range(3):
        ctx.qsg_sweep(2)
        ctx.qsg_tempering_swap()
        ctx.qsg_measure_correlators()
        for o in orcs:
            o.sweep(2)
            o.swap()
            o.measure()
    for gid, (s, o) in enumerate(zip(shapes, orcs)):
        assert np.array_equal(_gpu_spins(ctx, s, group=gid), o.spins())
        _check_corr(ctx.qsg_read_correlators(gid, raw=True), o.read())
        assert np.array_equal(ctx.qsg_read_accepts(gid), o.accepts())


def test_smallest_workload_full_run():
    """One sample, L=6, L_tau=32, k=0.29, 2 replicas, Metropolis, 2000 sweeps,
    correlators every 10 sweeps: everything bit-exact."""
    w = workloads.smallest()
    shape, lad = w.shapes[0], w.ladders[0]
    ctx, orc = _pair(shape, lad, seed=w.seed)
    for _ in range(w.total_sweeps // w.measure_every):
        ctx.qsg_sweep(w.measure_every)
        orc.sweep(w.measure_every)
        ctx.qsg_measure_correlators()
        orc.measure()
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    gpu = ctx.qsg_read_correlators(raw=True)
    _check_corr(gpu, orc.read())
    assert ctx.qsg_get_counters() == (2000, 0, 200)


def test_checkpoint_resume_is_bit_exact():
    shape = Q.Shape(8, 16, 64, 2, 3, Q.METROPOLIS, Q.PBC)
    lad = np.array([0.22, 0.28, 0.34])
    a = Q.Context([shape])
    a.qsg_init_samples(99, [lad])
    a.qsg_sweep(4)
    a.qsg_tempering_swap()
    state = a.qsg_get_spins(0)
    counters = a.qsg_get_counters()
    a.qsg_sweep(5)
    a.qsg_tempering_swap()
    b = Q.Context([shape])
    b.qsg_init_samples(99, [lad])
    b.qsg_set_spins(0, state)
    b.qsg_set_counters(*counters)
    b.qsg_sweep(5)
    b.qsg_tempering_swap()
    assert np.array_equal(a.qsg_get_spins(0), b.qsg_get_spins(0))


def _sampled_full_size(w, sweeps_before_swap, n_swaps, sample, configs, options=None):
    """Full-size GPU run against one sample simulated alone by the oracle."""
    shape, lad = w.shapes[0], w.ladders[0]
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(w.seed, [lad])
    for opt, val in (options or {}).items():
        ctx.qsg_set_option(opt, val)
    if options:
        # the graph batch must be what the sweeps replay
        assert sweeps_before_swap % options.get(Q.OPT_GRAPH, 1) == 0
    orc = oracle.OracleGroup(shape.L, shape.Ltau, 1, shape.n_replicas, shape.n_k, algo=shape.algo,
                             boundary=shape.boundary, first_sample=sample)
    orc.init(w.seed, lad)
    for _ in range(n_swaps):
        ctx.qsg_sweep(sweeps_before_swap)
        orc.sweep(sweeps_before_swap)
        ctx.qsg_tempering_swap()
        orc.swap()
    ctx.qsg_measure_correlators()
    words = ctx.qsg_get_spins(0).reshape(shape.words, shape.n_replicas, shape.n_k, -1)
    mine = (1 - 2 * ((words[sample // 64] >> np.uint64(sample % 64)) & np.uint64(1)).astype(np.int8))
    assert np.array_equal(mine.reshape(orc.spins()[0].shape), orc.spins()[0])
    assert np.array_equal(ctx.qsg_read_energies()[sample], orc.energies()[0])
    assert np.array_equal(ctx.qsg_read_accepts()[sample], orc.accepts()[0])
    gpu = ctx.qsg_read_correlators(raw=True)
    for r, j in configs:
        C, Qs = orc.measure_one(0, r, j)
        assert np.array_equal(gpu["C_raw"][r, sample, j], C)
        assert np.array_equal(gpu["Q2_raw"][r, sample, j], Qs)
    if options:
        ctx.qsg_set_option(Q.OPT_WAVEFRONT_VARIANT, 0)
    # properties that hold for every sample at any size
    assert np.all(gpu["C"][..., 0] == 1.0) and np.all(gpu["Q2"][..., 0] == 1.0)
    assert np.all(np.abs(gpu["C"]) <= 1.0) and np.all((gpu["Q2"] >= 0) & (gpu["Q2"] <= 1.0))
    assert np.all((gpu["q2"] >= 0) & (gpu["q2"] <= 1.0))


def test_mid_scale_sampled():
    w = workloads.mid_scale()
    _sampled_full_size(w, 10, 2, sample=37, configs=[(0, 0), (3, 23)])


def test_largest_sampled_in_bench_configuration():
    w = workloads.largest()
    _sampled_full_size(w, 2, 1, sample=77, configs=[(1, 5)])


def test_largest_sampled_with_the_benchmark_launch_options():
    """L = 24, L_tau = 2048, 128 samples x 4 replicas x 32 k, heat bath, in the
    launch configuration the benchmark times: one unit per block, chunks of 512
    planes with the last 32 slots in chunks of 128, and one CUDA-graph replay of
    30 sweeps, then a tempering step and a measurement; one sample against the
    oracle."""
    w = workloads.largest()
    options = {Q.OPT_CHUNK: 512, Q.OPT_TAIL: 32, Q.OPT_GRAPH: 30, Q.OPT_WAVEFRONT_VARIANT: 0}
    _sampled_full_size(w, 30, 1, sample=101, configs=[(2, 17)], options=options)


@pytest.mark.parametrize("L,Ltau,chunk", [(8, 16, 16), (8, 32, 16), (8, 64, 32), (8, 32, 0), (6, 32, 16),
                                          (24, 16, 16), (2, 16, 16), (32, 16, 16), (10, 48, 16), (4, 64, 0),
                                          (12, 48, 16), (16, 96, 32), (20, 32, 16)])
@pytest.mark.parametrize("algo,boundary", [(Q.METROPOLIS, Q.PBC), (Q.HEATBATH, Q.APBC)])
def test_wavefront_sweep_matches_oracle(L, Ltau, chunk, algo, boundary):
    """The fused one-pass sweep (chunked tau wavefront with deferred boundary
    planes) against the oracle, for several chunk lengths and block shapes."""
    shape = Q.Shape(L, Ltau, 70, 2, 2, algo, boundary)
    ctx, orc = _pair(shape, np.array([0.26, 0.32]), seed=31)
    ctx.qsg_set_option(Q.OPT_SWEEP_KERNEL, Q.SWEEP_WAVEFRONT)
    ctx.qsg_set_option(Q.OPT_CHUNK, chunk)
    for n in (1, 3):
        ctx.qsg_sweep(n)
        orc.sweep(n)
        assert np.array_equal(_gpu_spins(ctx, shape), orc.spins()), n
    ctx.qsg_tempering_swap()
    orc.swap()
    ctx.qsg_sweep(2)
    orc.sweep(2)
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())


@pytest.mark.parametrize("L,upb", [(8, 1), (8, 2), (8, 4), (8, 16), (12, 2), (16, 4), (4, 16)])
def test_units_per_block_of_the_generic_kernel_match_oracle(L, upb):
    """Grouping work units into blocks (QSG_OPT_UNITS_PER_BLOCK) changes no
    bit: every grouping, including ones rounded down to 512 threads, gives the
    oracle's spins; values that are not 0 or a power of two up to 16 are
    rejected."""
    shape = Q.Shape(L, 64, 70, 2, 3, Q.METROPOLIS, Q.APBC)
    ctx, orc = _pair(shape, workloads.uniform_ladder(0.22, 0.34, 3), seed=44)
    for bad in (-1, 3, 32):
        with pytest.raises(Q.QSGError):
            ctx.qsg_set_option(Q.OPT_UNITS_PER_BLOCK, bad)
    ctx.qsg_set_option(Q.OPT_SWEEP_KERNEL, Q.SWEEP_WAVEFRONT)
    ctx.qsg_set_option(Q.OPT_CHUNK, 16)
    ctx.qsg_set_option(Q.OPT_UNITS_PER_BLOCK, upb)
    for _ in range(2):
        ctx.qsg_sweep(3)
        orc.sweep(3)
        ctx.qsg_tempering_swap()
        orc.swap()
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    # and inside a captured graph
    ctx.qsg_set_option(Q.OPT_GRAPH, 4)
    ctx.qsg_sweep(4)
    orc.sweep(4)
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())


def test_reference_and_wavefront_kernels_agree_at_mid_scale():
    w = workloads.mid_scale()
    out = []
    for kern in (Q.SWEEP_REFERENCE, Q.SWEEP_WAVEFRONT):
        ctx = Q.Context(w.shapes)
        ctx.qsg_init_samples(w.seed, w.ladders)
        ctx.qsg_set_option(Q.OPT_SWEEP_KERNEL, kern)
        ctx.qsg_sweep(5)
        ctx.qsg_tempering_swap()
        ctx.qsg_sweep(5)
        out.append(ctx.qsg_get_spins(0))
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("L,R,algo", [(8, 2, Q.HEATBATH), (24, 2, Q.METROPOLIS), (24, 3, Q.HEATBATH),
                                      (20, 2, Q.HEATBATH), (20, 3, Q.METROPOLIS), (32, 2, Q.HEATBATH),
                                      (6, 4, Q.METROPOLIS)])
def test_wavefront_register_variants_match_oracle(variant, L, R, algo):
    """Every form of the wavefront kernel (one unit per block with two or four
    planes per barrier, the generic kernel) gives the oracle's bits."""
    shape = Q.Shape(L, 16, 70, R, 2, algo, Q.APBC)
    ctx, orc = _pair(shape, np.array([0.27, 0.3]), seed=41)
    ctx.qsg_set_option(Q.OPT_WAVEFRONT_VARIANT, variant)
    try:
        ctx.qsg_sweep(3)
        orc.sweep(3)
        assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    finally:
        ctx.qsg_set_option(Q.OPT_WAVEFRONT_VARIANT, 0)


@pytest.mark.parametrize("L,Ltau,boundary", [(10, 200, Q.APBC), (24, 130, Q.PBC), (6, 32, Q.APBC), (16, 256, Q.PBC),
                                             (12, 384, Q.APBC), (2, 4, Q.PBC), (32, 160, Q.APBC), (18, 96, Q.PBC),
                                             (20, 142, Q.APBC), (26, 64, Q.APBC), (28, 48, Q.PBC)])
def test_correlator_kernels_match_oracle(L, Ltau, boundary):
    """Tensor-core (tcgen05, FP8 +-1) and integer-pipe correlators both give the
    oracle's int64 sums: every chunk count of the tensor-core kernel (L^2 / 128
    rounded up: 1 .. 8), ragged tiles (L_tau not a multiple of 128; a single
    last column block), ragged K (L^2 not a multiple of 128), both boundary
    conditions, from three to six B stages in shared memory."""
    shape = Q.Shape(L, Ltau, 66, 2, 2, Q.HEATBATH, boundary)
    ctx, orc = _pair(shape, np.array([0.27, 0.31]), seed=55)
    ctx.qsg_sweep(3)
    orc.sweep(3)
    ctx.qsg_set_option(Q.OPT_CORR_KERNEL, Q.CORR_TENSOR)
    ctx.qsg_measure_correlators()
    ctx.qsg_set_option(Q.OPT_CORR_KERNEL, Q.CORR_INTEGER)
    ctx.qsg_measure_correlators()
    orc.measure()
    orc.measure()
    _check_corr(ctx.qsg_read_correlators(raw=True), orc.read())


@pytest.mark.parametrize("algo", [Q.METROPOLIS, Q.HEATBATH])
def test_persistent_ragged_launch_matches_oracle(algo):
    """Groups of different (L, L_tau) in one persistent launch per sweep, and
    on one stream each: every group's spins equal the oracle's and the
    sequential per-group launches'."""
    shapes = [Q.Shape(8, 32, 70, 2, 3, algo, Q.PBC), Q.Shape(12, 64, 5, 1, 2, algo, Q.APBC),
              Q.Shape(6, 16, 64, 2, 2, algo, Q.PBC), Q.Shape(16, 48, 3, 1, 1, algo, Q.PBC),
              Q.Shape(24, 32, 66, 1, 2, algo, Q.APBC)]
    lads = [np.array([0.2, 0.3, 0.4]), np.array([0.25, 0.33]), np.array([0.27, 0.28]), np.array([0.3]),
            np.array([0.26, 0.31])]
    results = []
    for mode in (2, 1, 3):  # persistent kernel, sequential, one stream per group
        ctx = Q.Context(shapes)
        ctx.qsg_init_samples(23, lads)
        ctx.qsg_set_option(Q.OPT_PERSISTENT, mode)
        for _ in range(3):
            ctx.qsg_sweep(2)
            ctx.qsg_tempering_swap()
        results.append([ctx.qsg_get_spins(gi) for gi in range(len(shapes))])
    for other in results[1:]:
        for a, b in zip(results[0], other):
            assert np.array_equal(a, b)
    for gid, (s, l) in enumerate(zip(shapes, lads)):
        o = oracle.OracleGroup(s.L, s.Ltau, s.n_samples, s.n_replicas, s.n_k, algo=s.algo, boundary=s.boundary,
                               group_id=gid)
        o.init(23, l)
        for _ in range(3):
            o.sweep(2)
            o.swap()
        assert np.array_equal(Q.unpack_spins(results[0][gid], s), o.spins()), gid


def test_ragged_workload_persistent_equals_per_group():
    w = workloads.ragged()
    out = []
    for mode in (2, 1, 3):
        ctx = Q.Context(w.shapes)
        ctx.qsg_init_samples(w.seed, w.ladders)
        ctx.qsg_set_option(Q.OPT_PERSISTENT, mode)
        ctx.qsg_sweep(3)
        out.append([ctx.qsg_get_spins(gi) for gi in range(len(w.shapes))])
        del ctx
        torch.cuda.empty_cache()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("persistent", [1, 2, 3])
def test_graph_replay_equals_direct_launches(persistent):
    """CUDA-graph replay of batches of sweeps gives the bits of direct launches
    and of the oracle, across replays, remainders, tempering steps, a counter
    restore and a recapture after an option change."""
    shapes = [Q.Shape(8, 32, 70, 2, 3, Q.HEATBATH, Q.PBC), Q.Shape(12, 64, 5, 1, 2, Q.HEATBATH, Q.APBC)]
    lads = [np.array([0.2, 0.3, 0.4]), np.array([0.25, 0.33])]

    def run(graph):
        ctx = Q.Context(shapes)
        ctx.qsg_init_samples(29, lads)
        ctx.qsg_set_option(Q.OPT_PERSISTENT, persistent)
        ctx.qsg_set_option(Q.OPT_GRAPH, graph)
        ctx.qsg_sweep(7)
        ctx.qsg_tempering_swap()
        ctx.qsg_sweep(5)
        ctx.qsg_set_option(Q.OPT_CHUNK, 16)
        ctx.qsg_sweep(6)
        sweeps, swaps, _ = ctx.qsg_get_counters()
        snap = [ctx.qsg_get_spins(gi) for gi in range(len(shapes))]
        ctx.qsg_sweep(3)
        ctx.qsg_set_counters(sweeps, swaps, -1)
        for gi, s in enumerate(snap):
            ctx.qsg_set_spins(gi, s)
        ctx.qsg_sweep(4)
        ctx.qsg_tempering_swap()
        return [ctx.qsg_get_spins(gi) for gi in range(len(shapes))]

    direct, graphed = run(0), run(3)
    for a, b in zip(direct, graphed):
        assert np.array_equal(a, b)
    for gid, (s, l) in enumerate(zip(shapes, lads)):
        o = oracle.OracleGroup(s.L, s.Ltau, s.n_samples, s.n_replicas, s.n_k, algo=s.algo, boundary=s.boundary,
                               group_id=gid)
        o.init(29, l)
        o.sweep(7)
        o.swap()
        o.sweep(5 + 6 + 4)
        o.swap()
        assert np.array_equal(Q.unpack_spins(graphed[gid], s), o.spins()), gid


def test_graph_replay_launch_count():
    shape = Q.Shape(8, 32, 64, 1, 2, Q.METROPOLIS, Q.PBC)
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(5, [np.array([0.3, 0.4])])
    ctx.qsg_set_option(Q.OPT_GRAPH, 4)
    ctx.qsg_sweep(4)  # capture, counter upload, one replay
    torch.cuda.synchronize()
    n0 = Q.qsg_kernel_launches()
    ctx.qsg_sweep(9)  # two replays of (4 sweeps + counter advance), one direct sweep
    torch.cuda.synchronize()
    assert Q.qsg_kernel_launches() - n0 == 2 * 5 + 1


def _close_nan(a, b, rtol=RTOL):
    a, b = np.asarray(a), np.asarray(b)
    both = np.isnan(a) & np.isnan(b)
    return np.all(both | (np.abs(a - b) <= rtol * np.maximum(np.abs(b), 1e-300)))


@pytest.mark.parametrize("L,Ltau,ns,R,K,boundary", [(6, 12, 70, 3, 2, Q.PBC), (8, 16, 64, 4, 2, Q.APBC),
                                                     (4, 8, 5, 2, 3, Q.PBC), (10, 8, 3, 9, 1, Q.PBC),
                                                     (2, 6, 64, 5, 2, Q.PBC)])
def test_onetime_observables_match_oracle(L, Ltau, ns, R, K, boundary):
    """Integer one-time sums bit for bit, FP64 per-sample and per-k values to
    1e-12 (R = 2: no triples; R = 9: beyond the three-replica limit)."""
    shape = Q.Shape(L, Ltau, ns, R, K, Q.HEATBATH, boundary)
    lad = np.linspace(0.25, 0.4, K)
    ctx, orc = _pair(shape, lad, seed=41)
    for _ in range(3):
        ctx.qsg_sweep(2)
        orc.sweep(2)
        ctx.qsg_tempering_swap()
        orc.swap()
        ctx.qsg_measure_correlators()
        orc.measure()
    got, ref = ctx.qsg_read_onetime(), orc.read_onetime()
    assert np.array_equal(got["raw"], ref["raw"])
    for f in Q.Context.ONETIME_SAMPLE_FIELDS:
        assert _close_nan(got[f], ref[f]), f
    for f in Q.Context.ONETIME_K_FIELDS:
        assert _close_nan(got["per_k"][f], ref["per_k"][f]), f
    if R < 3 or R > 8:
        assert np.all(np.isnan(got["chi3"]))
    else:
        assert np.all(np.isfinite(got["chi3"]))


def test_onetime_without_triples_keeps_pair_sums():
    shape = Q.Shape(8, 16, 64, 4, 2, Q.METROPOLIS, Q.PBC)
    outs = []
    for opt in (0, 1):
        ctx = Q.Context([shape])
        ctx.qsg_init_samples(43, [np.array([0.3, 0.35])])
        ctx.qsg_set_option(Q.OPT_ONETIME, opt)
        ctx.qsg_sweep(3)
        ctx.qsg_measure_correlators()
        outs.append(ctx.qsg_read_onetime())
        if opt == 1:
            with pytest.raises(Q.QSGError):
                ctx.qsg_set_option(Q.OPT_ONETIME, 0)  # after a measurement
    a, b = outs
    for f in ("q2", "q4", "chi2", "F2", "chi_lin"):
        assert np.array_equal(a[f], b[f])
    assert np.all(np.isnan(b["chi3"])) and np.all(np.isfinite(a["chi3"]))


def test_many_ladder_pairs_in_one_measurement_batch():
    """Short L_tau and many (word, k) pairs: the correlator batch is limited
    by the launch grid, not by the scratch; sampled samples match the oracle."""
    shape = Q.Shape(4, 16, 1024, 4, 32, Q.HEATBATH, Q.PBC)
    lad = np.linspace(0.2, 0.45, 32)
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(61, [lad])
    ctx.qsg_sweep(3)
    ctx.qsg_measure_correlators()
    got = ctx.qsg_read_correlators(raw=True)
    for b in (0, 517, 1023):
        o = oracle.OracleGroup(4, 16, 1, 4, 32, algo="heatbath", first_sample=b)
        o.init(61, lad)
        o.sweep(3)
        o.measure()
        ref = o.read()
        assert np.array_equal(got["C_raw"][:, b], ref["C_raw"][:, 0])
        assert np.array_equal(got["Q2_raw"][:, b], ref["Q2_raw"][:, 0])
        assert np.array_equal(got["q2_raw"][b], ref["q2_raw"][0])


@pytest.mark.parametrize("R", [128, 129, 1023])
def test_replica_counts_up_to_the_largest_match_oracle(R):
    """Up to 128 replicas (8,128 pairs) a block of the one-time pass keeps the
    per-pair Q^2 sums in shared memory; from 129 (8,256 pairs) up to the
    largest count a shape may have, 1023 (522,753 pairs), every slice adds
    them straight to the global sums.  Correlator and pair sums match the
    oracle bit for bit."""
    shape = Q.Shape(2, 4, 1, R, 1, Q.HEATBATH, Q.PBC)
    lad = np.array([0.3])
    ctx, orc = _pair(shape, lad, seed=R)
    ctx.qsg_sweep(2)
    orc.sweep(2)
    ctx.qsg_measure_correlators()
    orc.measure()
    _check_corr(ctx.qsg_read_correlators(raw=True), orc.read())
    assert np.array_equal(ctx.qsg_read_pair_overlaps(), orc.read_pair_overlaps())


def test_largest_ladder_matches_oracle():
    """128 k values (the largest ladder): 127 pairs per tempering step, the
    moves list up to 127 swapped pairs in batches of eight."""
    shape = Q.Shape(4, 8, 70, 2, 128, Q.METROPOLIS, Q.APBC)
    lad = workloads.uniform_ladder(0.2, 0.5, 128)
    ctx, orc = _pair(shape, lad, seed=17)
    for _ in range(4):
        ctx.qsg_sweep(2)
        orc.sweep(2)
        ctx.qsg_tempering_swap()
        orc.swap()
        assert np.array_equal(ctx.qsg_read_energies(), orc.energies())
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    assert np.array_equal(ctx.qsg_read_accepts(), orc.accepts())
    ctx.qsg_measure_correlators()
    orc.measure()
    _check_corr(ctx.qsg_read_correlators(raw=True), orc.read())


def test_longest_ltau_matches_oracle():
    """L_tau = 65,536 (the longest a shape may have): wavefront sweeps over
    1,024 chunks per slot, energies in 512 runs per slot, tempering steps."""
    shape = Q.Shape(4, 65536, 1, 2, 2, Q.HEATBATH, Q.APBC)
    lad = np.array([0.2998, 0.3])
    ctx, orc = _pair(shape, lad, seed=65)
    for _ in range(2):
        ctx.qsg_sweep(2)
        orc.sweep(2)
        ctx.qsg_tempering_swap()
        orc.swap()
        assert np.array_equal(ctx.qsg_read_energies(), orc.energies())
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())


@pytest.mark.parametrize("pinned", [False, True])
def test_correlator_readback_into_caller_buffers(pinned):
    """Reading into caller-owned (page-locked or pageable) buffers gives the
    same arrays as fresh ones; 70 samples leave padding bits in the second
    word, so every replica block is taken at its own offset."""
    shape = Q.Shape(6, 32, 70, 3, 2, Q.HEATBATH, Q.PBC)
    ctx, orc = _pair(shape, np.array([0.27, 0.31]), seed=9)
    ctx.qsg_sweep(2)
    orc.sweep(2)
    ctx.qsg_measure_correlators()
    orc.measure()
    ref = ctx.qsg_read_correlators(raw=True)
    _check_corr(ref, orc.read())
    out = ctx.correlator_buffers(pinned=pinned)
    for a in out.values():
        a.fill(np.nan)
    got = ctx.qsg_read_correlators(out=out)
    for k in ("C", "Q2", "q2"):
        assert got[k] is out[k]
        assert np.array_equal(got[k], ref[k])


def test_asynchronous_readback_is_ordered_before_the_next_measurement():
    """qsg_read_correlators_async queues the finish and copies and returns;
    a measurement and a second asynchronous read issued right after it must
    not overwrite the first read's sources before they are copied.  Both
    reads match the oracle after their own measurement, and a NULL copy
    stream is refused."""
    import torch
    shape = Q.Shape(6, 32, 70, 3, 2, Q.HEATBATH, Q.APBC)
    ctx, orc = _pair(shape, np.array([0.27, 0.31]), seed=13)
    copy_stream = torch.cuda.Stream()
    with pytest.raises(Q.QSGError):
        ctx.qsg_read_correlators_async(ctx.correlator_buffers(), 0)
    outs, refs = [], []
    for rep in range(2):
        ctx.qsg_sweep(2)
        orc.sweep(2)
        ctx.qsg_measure_correlators()
        orc.measure()
        refs.append(orc.read())
        out = ctx.correlator_buffers(pinned=True)
        for a in out.values():
            a.fill(np.nan)
        ctx.qsg_read_correlators_async(out, copy_stream)
        outs.append(out)
    ctx.qsg_wait_correlators()
    for out, ref in zip(outs, refs):
        for k in ("C", "Q2", "q2"):
            a, b = out[k], ref[k]
            both_nan = np.isnan(a) & np.isnan(b)
            assert np.all(both_nan | (np.abs(a - b) <= RTOL * np.maximum(np.abs(b), 1e-300))), k
    # the synchronous read after the asynchronous ones still agrees
    _check_corr(ctx.qsg_read_correlators(raw=True), refs[-1])
    ctx.qsg_wait_correlators()  # nothing pending: returns at once


@pytest.mark.parametrize("Ltau,chunk,tail", [(128, 64, 3), (128, 128, 12), (128, 64, 100), (1024, 512, 5)])
def test_wavefront_tail_slots_in_short_chunks_match_oracle(Ltau, chunk, tail):
    """The last `tail` slots swept in quarter-length chunks after every other
    unit (arrival counters at the finer spacing) give the oracle's bits; a
    tail longer than the group covers every slot."""
    shape = Q.Shape(8, Ltau, 70, 2, 3, Q.HEATBATH, Q.APBC)
    ctx, orc = _pair(shape, np.array([0.25, 0.3, 0.35]), seed=19)
    ctx.qsg_set_option(Q.OPT_CHUNK, chunk)
    ctx.qsg_set_option(Q.OPT_TAIL, tail)
    ctx.qsg_sweep(3)
    orc.sweep(3)
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    ctx.qsg_set_option(Q.OPT_TAIL, 0)
    ctx.qsg_sweep(2)
    orc.sweep(2)
    assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())


@pytest.mark.parametrize("L", [8, 12, 16, 20, 24])
@pytest.mark.parametrize("algo,boundary", [(Q.METROPOLIS, Q.APBC), (Q.HEATBATH, Q.PBC)])
@pytest.mark.parametrize("Ltau,chunk,tail,variant", [(16, 16, 0, 0), (64, 16, 0, 3), (64, 32, 0, 1),
                                                     (128, 64, 2, 0), (256, 128, 3, 1), (256, 64, 2, 3)])
def test_unit_kernel_chunks_and_tails_match_oracle(L, algo, boundary, Ltau, chunk, tail, variant):
    """The one-unit-per-block sweep (k_sweep_unit) against the oracle: single
    and several chunks per slot, tails swept in quarter-length chunks down to
    16 planes, two and four planes per barrier, both boundaries."""
    shape = Q.Shape(L, Ltau, 66, 2, 2, algo, boundary)
    ctx, orc = _pair(shape, np.array([0.26, 0.33]), seed=53)
    ctx.qsg_set_option(Q.OPT_WAVEFRONT_VARIANT, variant)
    try:
        ctx.qsg_set_option(Q.OPT_CHUNK, chunk)
        ctx.qsg_set_option(Q.OPT_TAIL, tail)
        for n in (1, 2):
            ctx.qsg_sweep(n)
            orc.sweep(n)
            assert np.array_equal(_gpu_spins(ctx, shape), orc.spins()), n
        ctx.qsg_tempering_swap()
        orc.swap()
        ctx.qsg_set_option(Q.OPT_GRAPH, 2)
        ctx.qsg_sweep(4)
        orc.sweep(4)
        assert np.array_equal(_gpu_spins(ctx, shape), orc.spins())
    finally:
        ctx.qsg_set_option(Q.OPT_WAVEFRONT_VARIANT, 0)


def test_device_buffer_checkpoint_resume_is_bit_exact():
    """qsg_get_spins_device / qsg_set_spins_device: the state through a device
    buffer equals the host copy, and resuming from it repeats the run bit for
    bit (the copies are ordered on the context's stream)."""
    shape = Q.Shape(24, 64, 70, 2, 3, Q.HEATBATH, Q.APBC)
    lad = np.array([0.25, 0.3, 0.35])
    ctx = Q.Context([shape])
    ctx.qsg_init_samples(12, [lad])
    ctx.qsg_sweep(3)
    ctx.qsg_tempering_swap()
    n = shape.slots * shape.Ltau * shape.L * shape.L
    saved = torch.empty(n, dtype=torch.int64, device=ctx.device)
    ctx.qsg_get_spins_device(0, saved)
    counters = ctx.qsg_get_counters()
    host = ctx.qsg_get_spins(0)
    assert np.array_equal(saved.cpu().numpy().view(np.uint64).reshape(host.shape), host)
    ctx.qsg_sweep(4)
    ctx.qsg_tempering_swap()
    first = ctx.qsg_get_spins(0)
    ctx.qsg_set_spins_device(0, saved)  # no host wait: ordered before the sweeps below
    ctx.qsg_set_counters(*counters)
    ctx.qsg_sweep(4)
    ctx.qsg_tempering_swap()
    assert np.array_equal(ctx.qsg_get_spins(0), first)
    with pytest.raises(Q.QSGError):
        ctx.qsg_set_spins_device(0, saved[:-1])


def test_ragged_workload_sampled_in_its_default_launch_form():
    """The ragged 640-sample workload (five groups, L = 8 .. 24, L_tau = 128 ..
    2048, uneven ladders, 6.47 GB) with one stream per group inside 6-sweep
    graphs: after two graph replays, a tempering step and one more replay,
    one sample of every group equals the oracle's run of that sample."""
    w = workloads.ragged()
    ctx = Q.Context(w.shapes)
    ctx.qsg_init_samples(w.seed, w.ladders)
    ctx.qsg_set_option(Q.OPT_PERSISTENT, 3)
    ctx.qsg_set_option(Q.OPT_GRAPH, 6)
    ctx.qsg_sweep(12)
    ctx.qsg_tempering_swap()
    ctx.qsg_sweep(6)
    for gid, (s, lad) in enumerate(zip(w.shapes, w.ladders)):
        sample = (37 * gid + 11) % s.n_samples
        orc = oracle.OracleGroup(s.L, s.Ltau, 1, s.n_replicas, s.n_k, algo=s.algo, boundary=s.boundary,
                                 group_id=gid, first_sample=sample)
        orc.init(w.seed, lad)
        orc.sweep(12)
        orc.swap()
        orc.sweep(6)
        words = ctx.qsg_get_spins(gid).reshape(s.words, s.n_replicas, s.n_k, -1)
        mine = (1 - 2 * ((words[sample // 64] >> np.uint64(sample % 64)) & np.uint64(1)).astype(np.int8))
        assert np.array_equal(mine.reshape(orc.spins()[0].shape), orc.spins()[0]), gid
        assert np.array_equal(ctx.qsg_read_accepts(gid)[sample], orc.accepts()[0]), gid
