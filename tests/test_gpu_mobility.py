"""GPU parity of the wall-RPY matvec (FP64 and FP32 multi-RHS kernels) and of
the blob geometry against the CPU oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import mobility as om, rigid
from paper_1709_02410_gb300 import F32, F64, synth

from gpu_util import DEV, handle_for, oracle_params, positions, rel2, to_dev

pytestmark = pytest.mark.gpu


def test_blob_geometry_matches_oracle():
    s = synth.boomerangs_1920()
    h = handle_for(s)
    r = h.blobs_from_bodies(to_dev(s.shape), to_dev(s.q), to_dev(s.theta)).cpu().numpy()
    np.testing.assert_allclose(r, positions(s), rtol=0, atol=1e-13)


@pytest.mark.parametrize("wall", [True, False])
def test_f64_matvec_c0(wall):
    s = synth.boomerangs_1920()
    r = positions(s)
    F = synth.gaussian(10, (3, s.n))
    h = handle_for(s, wall=wall)
    U = h.mobility_apply(to_dev(r), to_dev(F)).cpu().numpy()
    Uo = om.apply(r, F, oracle_params(s, wall))
    assert rel2(U, Uo) <= 1e-12


@pytest.mark.parametrize("n", [1, 2, 15, 17, 33, 129, 1000])
@pytest.mark.parametrize("k", [1, 3, 16])
def test_f64_matvec_ragged(n, k):
    """sizes below, at and across tile boundaries, penetrating blobs included"""
    rng = np.random.default_rng(n * 31 + k)
    box = max(2.0, np.sqrt(n) * 0.8)
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = rng.standard_normal((k, 3, n))
    s = synth.boomerangs_1920()
    h = handle_for(s)
    U = h.mobility_apply(to_dev(r), to_dev(F)).cpu().numpy()
    Uo = om.apply(r, F, oracle_params(s))
    assert rel2(U, Uo) <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 4, 8, 16])
def test_f32_matvec_c0(k):
    s = synth.boomerangs_1920()
    r = positions(s)
    F32in = synth.gaussian(20 + k, (k, 3, s.n), np.float32)
    h = handle_for(s)
    U = h.mobility_apply(to_dev(r), to_dev(F32in, torch.float32)).cpu().numpy()
    Uo = om.apply(r, F32in.astype(np.float64), oracle_params(s))
    for m in range(k):
        assert rel2(U[m], Uo[m]) <= 1e-5


@pytest.mark.parametrize("n", [1, 17, 65, 1000])
def test_f32_matvec_ragged(n):
    rng = np.random.default_rng(n)
    box = max(2.0, np.sqrt(n))
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = rng.standard_normal((5, 3, n)).astype(np.float32)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s))
    assert rel2(U, Uo) <= 1e-5


def test_mixed_mode_f32_pairs_f64_vectors():
    s = synth.boomerangs_1920()
    r = positions(s)
    F = synth.gaussian(30, (3, s.n))
    h = handle_for(s)
    U = h.mobility_apply(to_dev(r), to_dev(F), dtype=F32).cpu().numpy()
    assert rel2(U, om.apply(r, F, oracle_params(s))) <= 1e-5


def test_empty_is_noop():
    s = synth.boomerangs_1920()
    h = handle_for(s)
    r = torch.zeros((3, 0), dtype=torch.float64, device=DEV)
    F = torch.zeros((3, 0), dtype=torch.float64, device=DEV)
    U = h.mobility_apply(r, F)
    assert U.numel() == 0


@pytest.mark.parametrize("k", [1, 2, 16])
def test_f32_full_size_row_sampled(k):
    """65,535 blobs in the bench's launch configurations (k = 1, 2: packed
    symmetric kernel; k = 16: one-direction kernel); 128 sampled target rows
    (the first and last blob included) against the oracle."""
    s = synth.boomerangs_65535()
    r = positions(s)
    F = synth.gaussian(40 + k, (k, 3, s.n), np.float32)
    h = handle_for(s)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    rows = np.random.default_rng(41).choice(s.n, 128, replace=False)
    rows[0], rows[1] = 0, s.n - 1
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s), rows=rows)
    assert rel2(U[:, :, rows], Uo) <= 1e-5


def test_f64_full_size_row_sampled():
    s = synth.boomerangs_65535()
    r = positions(s)
    F = synth.gaussian(42, (3, s.n))
    h = handle_for(s)
    U = h.mobility_apply(to_dev(r), to_dev(F)).cpu().numpy()
    rows = np.random.default_rng(43).choice(s.n, 64, replace=False)
    Uo = om.apply(r, F, oracle_params(s), rows=rows)
    assert rel2(U[:, rows], Uo) <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 4])
@pytest.mark.parametrize("n", [5, 129, 1000])
def test_f32_symmetric_and_one_direction_agree(k, n):
    """the symmetric kernel (default for k <= 4) and the one-direction kernel"""
    rng = np.random.default_rng(7 * n + k)
    box = max(2.0, np.sqrt(n))
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = rng.standard_normal((k, 3, n)).astype(np.float32)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    U1 = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    h.set_symmetric(False)
    U2 = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s))
    assert rel2(U1, Uo) <= 1e-5 and rel2(U2, Uo) <= 1e-5


def test_autotune_picks_a_correct_kernel():
    s = synth.boomerangs_1920()
    r = positions(s)
    F = synth.gaussian(60, (1, 3, s.n), np.float32)
    h = handle_for(s)
    choice, ms = h.autotune(to_dev(r), 1)
    assert 0 <= choice <= 6 and ms > 0
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5
    for v in range(6):
        h.set_symmetric(True)
        h.set_sym_variant(v)
        U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
        assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5


def test_autotune_classes_are_independent():
    """Autotuning k = 2 keeps the k = 1 choice; both classes stay correct."""
    s = synth.boomerangs_1920()
    r = positions(s)
    h = handle_for(s)
    c1, _ = h.autotune(to_dev(r), 1)
    c2, _ = h.autotune(to_dev(r), 2)
    assert 0 <= c1 <= 6 and 0 <= c2 <= 6
    for k in (1, 2, 3):
        F = synth.gaussian(61 + k, (k, 3, s.n), np.float32)
        U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
        assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5


def test_fma_peak_probe():
    """The FMA-throughput probe returns a plausible figure: below the nominal
    dense peaks (FP32: 152 SMs x 128 lanes x 2 x 2.07 GHz) with margin, and
    FP32 well above FP64."""
    h = handle_for(synth.boomerangs_1920())
    f32 = h.measure_fma_peak(F32)
    f64 = h.measure_fma_peak(F64)
    f32v = h.measure_fma_peak(3)   # packed FMAs reading three distinct varying registers
    assert 1.0 < f32 < 1.2 * 80.55
    assert 0.0 < f64 < f32
    assert 0.0 < f32v < f32


@pytest.mark.parametrize("variant", [-1, 4, 5])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 31, 255, 256, 257, 700, 2049, 4500])
def test_f32_packed_symmetric_kernel(k, n, variant):
    """The packed symmetric kernel (256-blob home tiles, two-wide FP32
    arithmetic; two home blobs per thread by default, four in variants 4 and
    5) against the oracle and against the one-home symmetric kernel: sizes
    below, at and across the 256-blob tile and the 2048-visitor chunk, blobs
    overlapping each other and the wall."""
    rng = np.random.default_rng(11 * n + k)
    box = max(2.0, np.sqrt(n))
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = rng.standard_normal((k, 3, n)).astype(np.float32)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    h.set_sym_variant(variant)
    Up = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    h.set_packed(False)
    Us = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s))
    assert rel2(Up, Uo) <= 1e-5 and rel2(Us, Uo) <= 1e-5
    assert rel2(Up, Us) <= 1e-5


@pytest.mark.parametrize("k", [1, 2, 4])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_f32_packed_variants(variant, k):
    s = synth.boomerangs_1920()
    r = positions(s)
    F = synth.gaussian(70 + variant, (k, 3, s.n), np.float32)
    h = handle_for(s)
    h.set_sym_variant(variant)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 257, 2049, 9000])
def test_f32_packed_symmetric_fixed_point_and_partials(k, n):
    """The packed symmetric kernel's two accumulations: fixed point per blob
    (the default; integer atomics) and per-home-tile partials with the
    fixed-order reduction.  Both against the oracle, against each other (they
    sum the same FP32 tile sums, to ~1e-12 and to ~48 bits, so they differ by
    FP32 output rounding), and each bit for bit against a repeat of itself."""
    rng = np.random.default_rng(13 * n + k)
    box = max(2.0, np.sqrt(n))
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = rng.standard_normal((k, 3, n)).astype(np.float32)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    rd, Fd = to_dev(r), to_dev(F, torch.float32)
    Ufx = h.mobility_apply(rd, Fd).cpu().numpy()
    assert np.array_equal(Ufx, h.mobility_apply(rd, Fd).cpu().numpy())
    Ufx64 = h.mobility_apply(rd, to_dev(F.astype(np.float64)), dtype=1).cpu().numpy()
    h.set_sym_partials(True)
    Upt = h.mobility_apply(rd, Fd).cpu().numpy()
    assert np.array_equal(Upt, h.mobility_apply(rd, Fd).cpu().numpy())
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s))
    assert rel2(Ufx, Uo) <= 1e-5 and rel2(Ufx64, Uo) <= 1e-5 and rel2(Upt, Uo) <= 1e-5
    assert rel2(Ufx, Upt) <= 1e-6


def test_f32_fixed_point_wide_force_range():
    """Forces over ten decades (log-uniform 1e-4..1e4, one blob at 1e6): the
    fixed-point step 2^-S is set by the largest force, so small rows carry an
    absolute error of at most (contributions per blob) x 2^-S / 2, in units of
    1 / (8 pi eta a).  Checked element by element against the partials path
    (the same FP32 tile sums, no fixed-point rounding), and both against the
    oracle."""
    n = 9000
    rng = np.random.default_rng(4242)
    box = np.sqrt(n)
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = rng.standard_normal((1, 3, n)) * 10.0 ** rng.uniform(-4, 4, n)
    F[0, :, 4321] = [1e6, -1e6, 5e5]
    F = F.astype(np.float32)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    rd, Fd = to_dev(r), to_dev(F, torch.float32)
    Ufx = h.mobility_apply(rd, Fd).cpu().numpy().astype(np.float64)
    h.set_sym_partials(True)
    Upt = h.mobility_apply(rd, Fd).cpu().numpy().astype(np.float64)
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s))
    assert rel2(Ufx, Uo) <= 1e-5 and rel2(Upt, Uo) <= 1e-5
    # S as the kernel takes it: 2^S = 2^61 / 2^e with 4 n max|F| < 2^e
    bound = 4.0 * n * float(np.abs(F).max())
    step = 2.0 ** -(61 - np.frexp(bound)[1])
    contributions = n // 256 + n // 32 + 2      # visitor tiles before the blob + its home items
    abs_tol = contributions * step / 2 / (8 * np.pi * synth.ETA * s.a)
    assert np.all(np.abs(Ufx - Upt) <= 4 * np.finfo(np.float32).eps * np.abs(Upt) + abs_tol)


@pytest.mark.parametrize("n,scale", [(2049, 1e-30), (2049, 1e-20), (2049, 1e20), (9000, 4e33)])
def test_f32_fixed_point_extreme_force_scales(n, scale):
    """The fixed-point exponent follows the forces' scale over the FP32 range:
    forces of 1e-30 (2^S = 2^145, beyond FP32's largest power of two) and of
    4e33 at 9,000 blobs (4 n max|F| ~ 6e38, beyond FP32's largest value) give
    the oracle's velocities to the FP32 tolerance, as N(0,1) forces do.  (Far
    smaller forces meet FP32's flush of subnormal products, not the fixed
    point.)"""
    rng = np.random.default_rng(977)
    box = np.sqrt(n)
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = (rng.standard_normal((2, 3, n)) * scale).astype(np.float32)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(U))
    assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5


def test_f32_fixed_point_non_finite_input_gives_nan():
    """A NaN force or position makes the fixed-point sums NaN, as the
    fixed-order reduction's sums would be."""
    s = synth.boomerangs_1920()
    r = positions(s)
    F = synth.gaussian(3, (1, 3, s.n), np.float32)
    h = handle_for(s)
    Fb = F.copy()
    Fb[0, 1, 77] = np.nan
    assert np.isnan(h.mobility_apply(to_dev(r), to_dev(Fb, torch.float32)).cpu().numpy()).any()
    rb = r.copy()
    rb[0, 5] = np.nan
    assert np.isnan(h.mobility_apply(to_dev(rb), to_dev(F, torch.float32)).cpu().numpy()).any()
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()   # and the handle is fine
    assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_f32_one_direction_packed_tile(k):
    """With the symmetric kernel off, k = 1, 3, 4 run on the packed tile (two
    targets per thread; one system of the batched kernel) and k = 2 on its
    own tile; packed and unpacked one-direction kernels against the oracle at
    sizes across the 64-source tile and the 2048-source chunk, the work list
    rebuilt as n changes, FP32 and FP64 vectors."""
    s = synth.boomerangs_1920()
    h = handle_for(s)
    h.set_symmetric(False)
    for n in (1, 63, 129, 2049, 4500, 700):
        rng = np.random.default_rng(13 * n + k)
        box = max(2.0, np.sqrt(n))
        r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
        F = rng.standard_normal((k, 3, n)).astype(np.float32)
        Uo = om.apply(r, F.astype(np.float64), oracle_params(s))
        h.set_packed(True)
        Up = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
        Ud = h.mobility_apply(to_dev(r), to_dev(F.astype(np.float64)), dtype=F32).cpu().numpy()
        h.set_packed(False)
        Uu = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
        assert rel2(Up, Uo) <= 1e-5 and rel2(Ud, Uo) <= 1e-5 and rel2(Uu, Uo) <= 1e-5, n


@pytest.mark.parametrize("sym", [True, False])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_f32_half_million_blobs_row_sampled(k, sym):
    """500,010 blobs (33,334 boomerangs at the same density): the packed
    symmetric kernel with its fixed-point accumulation (memory O(n)); with the
    symmetric kernel off, the one-direction kernels (k = 2 its own tile, k = 1,
    3 the packed tile); 32 sampled rows against the oracle."""
    nb = 33334
    s = synth.boomerang_suspension(nb, 40.0 * np.sqrt(nb / 128), 44)
    r = positions(s)
    F = synth.gaussian(45 + k, (k, 3, s.n), np.float32)
    h = handle_for(s)
    h.set_symmetric(sym)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    rows = np.random.default_rng(46).choice(s.n, 32, replace=False)
    rows[0], rows[1] = 0, s.n - 1
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s), rows=rows)
    h.close()
    assert rel2(U[:, :, rows], Uo) <= 1e-5


@pytest.mark.parametrize("k", [1, 2])
def test_f32_packed_far_from_origin_and_wide(k):
    """Positions far from the origin and spread wide: the FP32 kernels carry
    x, y as hi/lo float pairs, so a translation by 10^5 a leaves U unchanged
    (to FP32 rounding of the pair blocks), and a 4,000 a wide scatter of
    clusters still meets the oracle at 1e-5."""
    s = synth.boomerangs_1920()
    r = positions(s)
    F = synth.gaussian(47 + k, (k, 3, s.n), np.float32)
    h = handle_for(s)
    U0 = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    rt = r.copy()
    rt[0] += 1.0e5 * s.a
    rt[1] -= 3.0e5 * s.a
    Ut = h.mobility_apply(to_dev(rt), to_dev(F, torch.float32)).cpu().numpy()
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s))
    assert rel2(U0, Uo) <= 1e-5 and rel2(Ut, Uo) <= 1e-5 and rel2(Ut, U0) <= 1e-6
    # bodies in 16 clusters spread over 4,000 a
    rng = np.random.default_rng(48)
    shift = rng.uniform(-2000.0, 2000.0, (16, 2)) * s.a
    rw = r.copy()
    body = np.arange(s.n) // s.nper
    rw[0] += shift[body % 16, 0]
    rw[1] += shift[body % 16, 1]
    Uw = h.mobility_apply(to_dev(rw), to_dev(F, torch.float32)).cpu().numpy()
    assert rel2(Uw, om.apply(rw, F.astype(np.float64), oracle_params(s))) <= 1e-5


@pytest.mark.parametrize("k", [1, 8, 16])
@pytest.mark.parametrize("n", [1, 700, 4500])
def test_f32_one_direction_fixed_point_and_partials(k, n):
    """The one-direction FP32 kernel's two accumulations: fixed point per blob
    (the default) and per-chunk partials with the fixed-order reduction.  Both
    against the oracle, against each other (the same FP32 chunk sums), and
    each bit for bit against a repeat of itself; the fixed point in the
    periodic cell as well."""
    rng = np.random.default_rng(17 * n + k)
    box = max(2.0, np.sqrt(n))
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = rng.standard_normal((k, 3, n)).astype(np.float32)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    h.set_symmetric(False)
    rd, Fd = to_dev(r), to_dev(F, torch.float32)
    Ufx = h.mobility_apply(rd, Fd).cpu().numpy()
    assert np.array_equal(Ufx, h.mobility_apply(rd, Fd).cpu().numpy())
    h.set_sym_partials(True)
    Upt = h.mobility_apply(rd, Fd).cpu().numpy()
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s))
    assert rel2(Ufx, Uo) <= 1e-5 and rel2(Upt, Uo) <= 1e-5
    assert rel2(Ufx, Upt) <= 1e-6
    if k == 16:
        from paper_1709_02410_gb300 import Handle
        L = max(4.0, box)
        hp = Handle(synth.ETA, s.a, synth.KT, Lx=L, Ly=L)
        Up = hp.mobility_apply(rd, Fd).cpu().numpy()
        assert rel2(Up, om.apply(r, F.astype(np.float64), om.Params(synth.ETA, s.a, Lx=L, Ly=L))) <= 1e-5


def test_f32_one_direction_fixed_point_extreme_scale_and_nan():
    """k = 8 (one-direction kernel): forces of 4e33 at 9,000 blobs (4 n max|F|
    beyond FP32's range) match the oracle; a NaN force gives NaN."""
    n = 9000
    rng = np.random.default_rng(979)
    box = np.sqrt(n)
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = (rng.standard_normal((8, 3, n)) * 4e33).astype(np.float32)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(U))
    assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5
    F[3, 2, 10] = np.nan
    assert np.isnan(h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()).any()
