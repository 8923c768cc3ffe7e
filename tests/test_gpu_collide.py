"""Parity of the CUDA collision operator with the FP64 oracle (C ABI calls).

Plain FP64 form: <= 1e-12 relative L2 against the oracle, and element by
element.  FP32 form, against the oracle on the same FP32-rounded input:
  * on the shifted-Maxwellian workload (Mach 0-3) the target of the mixed
    form, rel-L2 <= 1e-6 over all cells and velocities (TARGET32);
  * in every FP32 case, every cell within the bounds derived from the
    rounding count (gpu_util.fp32_cell_bounds): its L2 error and each
    element's error against u times the cell's absolute mode sum, which a
    localised defect (a wrong weight row, a wrong mode, a wrong cell of a
    ragged tile) exceeds by orders of magnitude;
  * TOL32 = 1e-5 rel-L2 only where the inputs carry 5 % point noise or 48^2 /
    3-D grids: there the FP32 floor itself (FP32 spectra, products and
    accumulation under the gain/loss cancellation) is 1e-6 to 4e-6, above the
    target; the FP32X2 form is the one that meets 1e-6 there.
"""
import numpy as np
import pytest

from paper_2103_14890_gb300 import workloads
from gpu_util import AbsModeSum, as_input, bz_module, check_fp32_cells, relerr, to_dev

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5
TARGET32 = 1e-6


@pytest.fixture(scope="module")
def bz():
    return bz_module()


@pytest.fixture(scope="module")
def oracle_k():
    import oracle
    cache = {}

    def get(dim, N, L, gamma):
        key = (dim, N, L, gamma)
        if key not in cache:
            cache[key] = oracle.Kernel(dim, N, L, gamma)
        return cache[key]
    return get


def _gpu_collide(bz, dim, N, L, gamma, f, precision, conserve=False):
    g = bz.Grid(dim, N, L)
    m = bz.Modes(g, gamma)
    Q = bz.collide_batch(m, to_dev(f, precision), precision=precision, conserve=conserve)
    bz.check()
    return Q.double().cpu().numpy()


@pytest.mark.parametrize("dim,N,gamma", [(2, 8, 0.0), (2, 16, 1.0), (3, 6, 1.0)])
def test_kernel_modes_match_oracle(bz, oracle_k, dim, N, gamma):
    m = bz.Modes(bz.Grid(dim, N, 8.0), gamma)
    got = m.beta_table()
    k = oracle_k(dim, N, 8.0, gamma)
    want = k.beta_table()
    # the library zeroes entries with l + m outside K_h; compare where it does not
    mask = got != 0
    assert np.abs(got - want)[mask].max() < 1e-13 * np.abs(want).max()
    assert np.abs(want[~mask][np.abs(want[~mask]) > 0]).size >= 0


def test_fast_kernels_selected(bz):
    """The register-blocked FP32 mode sum serves every 2-D grid with 16 <= N <= 48
    and the 3-D grids up to 16^3 (a silent fall back to the generic kernel would
    hide a table-building bug)."""
    for N in (16, 24, 32):
        assert bz.Modes(bz.Grid(2, N, 10.0), 1.0).modesum_variant >= 1, N
    assert bz.Modes(bz.Grid(2, 48, 10.0), 1.0).modesum_variant in (3, 8, 9, 10)    # only 16-cell tiles fit
    assert bz.Modes(bz.Grid(3, 16, 10.0), 1.0).modesum_variant == 4    # 8-cell tiles, 3-D rows
    assert bz.Modes(bz.Grid(3, 8, 8.0), 1.0).modesum_variant >= 1   # 16-wide blocks overhang a 7-mode row
    assert bz.Modes(bz.Grid(2, 64, 10.0), 1.0).modesum_variant == 0


@pytest.mark.parametrize("dim,N,variant", [(2, N, v) for N in (16, 24, 32) for v in (1, 2, 3, 5, 6, 7, 8, 9, 10)]
                         + [(2, 16, 4), (3, 8, 1), (3, 8, 2), (3, 8, 3), (3, 8, 5), (3, 8, 6), (3, 8, 7),
                            (2, 48, 3), (2, 48, 8), (2, 48, 9), (2, 48, 10)])
def test_fp32_each_kernel_variant(bz, oracle_k, monkeypatch, dim, N, variant):
    """Every register-blocked variant (fixed through BZ_MODESUM_VARIANT, bypassing
    the autotuner) against the oracle: 70 cells = 2 full tiles and a ragged tail."""
    monkeypatch.setenv("BZ_MODESUM_VARIANT", str(variant))
    L = 10.0
    m = bz.Modes(bz.Grid(dim, N, L), 1.0)
    assert m.modesum_variant == variant
    f = workloads.bi_maxwellian(70, dim, N, L, seed=1100 + N)
    fin = as_input(f, "fp32")
    Q = bz.collide_batch(m, to_dev(f, "fp32"), precision="fp32")
    bz.check()
    k = oracle_k(dim, N, L, 1.0)
    Qr = k.collide(fin)
    Qg = Q.double().cpu().numpy()
    assert relerr(Qg, Qr) < TOL32
    check_fp32_cells(k, fin, Qg, Qr, what="variant %d N=%d d=%d" % (variant, N, dim))


_SPLIT_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2103_14890_gb300 import binding as bz, workloads
variant, extra = int(sys.argv[2]), int(sys.argv[3])
N, L = 32, 10.0
sms = torch.cuda.get_device_properties(0).multi_processor_count
n = sms * 32 + extra
f = workloads.bi_maxwellian(n, 2, N, L, seed=1500)
m = bz.Modes(bz.Grid(2, N, L), 1.0)            # the cached choice: timed path, split allowed
assert m.modesum_variant == variant, m.modesum_variant
Q = bz.collide_batch(m, torch.tensor(f, dtype=torch.float32, device="cuda")).cpu().numpy()
import os
os.environ["BZ_MODESUM_VARIANT"] = str(variant)
m_main = bz.Modes(bz.Grid(2, N, L), 1.0)
os.environ["BZ_MODESUM_VARIANT"] = sys.argv[4]
m_tail = bz.Modes(bz.Grid(2, N, L), 1.0)
Qa = bz.collide_batch(m_main, torch.tensor(f[:sms * 32], dtype=torch.float32, device="cuda")).cpu().numpy()
Qb = bz.collide_batch(m_tail, torch.tensor(f[sms * 32:], dtype=torch.float32, device="cuda")).cpu().numpy()
bz.check()
assert np.array_equal(Q[:sms * 32], Qa)
assert np.array_equal(Q[sms * 32:], Qb)
print("ok")
"""


def test_paired_variants_need_half_row_blocks(bz, monkeypatch):
    """The paired-orientation variants (8, 9, 10) compute k_2 < 0 in the
    mirrored half of each task, which needs output blocks of k_2 >= 0 only
    (8 outputs <= h + 1): on 8^3 (h = 3) they are not built and a request for
    one falls back to the autotuner's choice."""
    for v in (8, 9, 10):
        monkeypatch.setenv("BZ_MODESUM_VARIANT", str(v))
        assert bz.Modes(bz.Grid(3, 8, 8.0), 1.0).modesum_variant not in (8, 9, 10)
        assert bz.Modes(bz.Grid(2, 16, 8.0), 1.0).modesum_variant == v


@pytest.mark.parametrize("variant", [1, 7])
@pytest.mark.parametrize("extra", [70, 30 * 32 + 5, 50 * 32, 100 * 32 - 1])
def test_last_wave_split_is_exact(tmp_path, variant, extra):
    """A 32-cell variant chosen as the autotuner would (through the tune cache,
    in a fresh process): whole waves of CTAs run one tile each and the tiles of
    the last partial wave are split over 8, 4 or 2 CTAs (3, 31, 50 extra
    tiles) or, beyond half the SMs (100 extra tiles), run on the 16-cell
    variant when that one sums every output in the same order (the scalar
    one-cell-per-lane variants), else as a plain partial wave: every cell must
    equal a run of a fixed variant (cells are independent)."""
    import os
    import subprocess
    import sys
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cache = tmp_path / "tune.txt"
    cache.write_text("2 32 %d %d\n" % (sms, variant))
    tail = str(variant) if variant == 7 or extra < 100 * 32 - 1 else "3"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, BZ_TUNE_CACHE=str(cache))
    env.pop("BZ_MODESUM_VARIANT", None)
    r = subprocess.run([sys.executable, "-c", _SPLIT_CHILD, root, str(variant), str(extra), tail], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


@pytest.mark.parametrize("n", [1, 8, 13])
def test_fp32_3d_16_grid_8_cell_tiles(bz, oracle_k, n):
    """16^3 grid on [-10,10]^3 (register-blocked 3-D path, 8-cell tiles): one
    cell, exactly one CTA, and one and a half CTAs, against the oracle."""
    N, L = 16, 10.0
    m = bz.Modes(bz.Grid(3, N, L), 1.0)
    assert m.modesum_variant == 4
    f = workloads.bi_maxwellian(n, 3, N, L, seed=1400 + n)
    fin = as_input(f, "fp32")
    Q = bz.collide_batch(m, to_dev(f, "fp32"), precision="fp32")
    bz.check()
    k = oracle_k(3, N, L, 1.0)
    Qr = k.collide(fin)
    Qg = Q.double().cpu().numpy()
    assert relerr(Qg, Qr) < TOL32
    check_fp32_cells(k, fin, Qg, Qr, what="16^3 n=%d" % n)


@pytest.mark.parametrize("n", [1, 16, 17, 45])
def test_fp32_48_grid_16_cell_tiles(bz, oracle_k, n):
    """48^2 grid on [-10,10]^2 (16-cell tiles, the timed variant): single cell,
    exactly one CTA, one past it, and a ragged 32-cell tile pair, against the
    oracle."""
    N, L = 48, 10.0
    m = bz.Modes(bz.Grid(2, N, L), 1.0)
    assert m.modesum_variant in (3, 8, 9, 10)
    f = workloads.bi_maxwellian(n, 2, N, L, seed=1200 + n)
    fin = as_input(f, "fp32")
    Q = bz.collide_batch(m, to_dev(f, "fp32"), precision="fp32")
    bz.check()
    k = oracle_k(2, N, L, 1.0)
    Qr = k.collide(fin)
    Qg = Q.double().cpu().numpy()
    assert relerr(Qg, Qr) < TOL32
    check_fp32_cells(k, fin, Qg, Qr, what="48^2 n=%d" % n)


def test_fp64_small_config_matches_oracle(bz, oracle_k):
    """64 cells, 16^2 grid on [-8,8]^2, Maxwell molecules, bi-Maxwellians."""
    f = workloads.bi_maxwellian(64, 2, 16, 8.0, seed=1001)
    Q = _gpu_collide(bz, 2, 16, 8.0, 0.0, f, "fp64")
    Qr = oracle_k(2, 16, 8.0, 0.0).collide(f)
    assert relerr(Q, Qr) < TOL64
    assert np.abs(Q - Qr).max() < TOL64 * np.abs(Qr).max()


def test_fp64_ragged_tiles_hard_spheres(bz, oracle_k):
    """100 cells (3 full 32-cell tiles + a tail of 4), 32^2 on [-10,10]^2, VHS, noise."""
    f = workloads.bi_maxwellian(100, 2, 32, 10.0, seed=1002, noise=0.05)
    Q = _gpu_collide(bz, 2, 32, 10.0, 1.0, f, "fp64")
    Qr = oracle_k(2, 32, 10.0, 1.0).collide(f)
    assert relerr(Q, Qr) < TOL64
    for c in (0, 31, 32, 95, 96, 99):
        assert relerr(Q[c], Qr[c]) < 10 * TOL64


def test_fp64_conservation_fix(bz, oracle_k):
    f = workloads.shifted_maxwellians(37, 2, 32, 10.0, seed=5)
    Q = _gpu_collide(bz, 2, 32, 10.0, 1.0, f, "fp64", conserve=True)
    Qr = oracle_k(2, 32, 10.0, 1.0).collide(f, conserve=True)
    assert relerr(Q, Qr) < TOL64
    v = workloads.velocity_nodes(32, 10.0)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    for p in (np.ones_like(V1), V1, V2, V1 ** 2 + V2 ** 2):
        mom = Q @ p.ravel()
        assert np.abs(mom).max() < 1e-12 * np.abs(Q).sum(axis=1).max() * np.abs(p).max()


@pytest.mark.parametrize("N,n", [(16, 33), (24, 40), (32, 37), (48, 21)])
def test_fp32_conservation_fix_every_tile_fft(bz, oracle_k, N, n):
    """FP32 form with BZ_CONSERVE on every grid the tile FFT kernels serve
    (the 48^2 epilogue reduces each cell's moments over two warps): against
    the oracle's projected Q, and moments of 1, v, |v|^2 at FP32 level."""
    L = 10.0
    f = workloads.bi_maxwellian(n, 2, N, L, seed=1300 + N)
    Q = _gpu_collide(bz, 2, N, L, 1.0, f, "fp32", conserve=True)
    Qr = oracle_k(2, N, L, 1.0).collide(as_input(f, "fp32"), conserve=True)
    assert relerr(Q, Qr) < TOL32
    v = workloads.velocity_nodes(N, L)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    for p in (np.ones_like(V1), V1, V2, V1 ** 2 + V2 ** 2):
        mom = Q @ p.ravel()
        assert np.abs(mom).max() < 1e-5 * np.abs(Q).sum(axis=1).max() * np.abs(p).max()


@pytest.mark.parametrize("N,n", [(24, 9), (48, 5), (48, 13)])
@pytest.mark.parametrize("conserve", [False, True])
def test_fp64_mixed_radix_fft_grids(bz, oracle_k, N, n, conserve):
    """FP64 form on the grids whose tile FFTs are mixed radix (24 = 3 x 8,
    48 = 3 x 16; 48^2 mode sums on the generic kernel) against the oracle."""
    L = 10.0
    f = workloads.bi_maxwellian(n, 2, N, L, seed=1600 + N)
    Q = _gpu_collide(bz, 2, N, L, 1.0, f, "fp64", conserve=conserve)
    Qr = oracle_k(2, N, L, 1.0).collide(f, conserve=conserve)
    assert relerr(Q, Qr) < TOL64


def test_fp64_three_dimensional(bz, oracle_k):
    f = workloads.bi_maxwellian(35, 3, 8, 8.0, seed=11)
    Q = _gpu_collide(bz, 3, 8, 8.0, 1.0, f, "fp64")
    Qr = oracle_k(3, 8, 8.0, 1.0).collide(f)
    assert relerr(Q, Qr) < TOL64


@pytest.mark.parametrize("seed,kind", [(1003, "shifted"), (1002, "noise")])
def test_fp32_matches_oracle(bz, oracle_k, seed, kind):
    """70 cells (2 full tiles and a ragged tail) of the benchmark's workload
    (shifted Maxwellians, Mach 0-3): the mixed form's 1e-6 target.  The 5 %
    noise inputs of the 4096-cell configuration sit above it in FP32 (below
    target: their FP32 floor is ~2.5e-6) and are held to the per-cell bounds
    and TOL32."""
    if kind == "shifted":
        f = workloads.shifted_maxwellians(70, 2, 32, 10.0, seed=seed)
    else:
        f = workloads.bi_maxwellian(70, 2, 32, 10.0, seed=seed, noise=0.05)
    Q = _gpu_collide(bz, 2, 32, 10.0, 1.0, f, "fp32")
    fin = as_input(f, "fp32")
    k = oracle_k(2, 32, 10.0, 1.0)
    Qr = k.collide(fin)
    err = relerr(Q, Qr)
    print("fp32 %s rel-L2 %.3e" % (kind, err))
    assert err < (TARGET32 if kind == "shifted" else TOL32)
    check_fp32_cells(k, fin, Q, Qr, what="fp32 " + kind)


def test_fp32_three_dimensional(bz, oracle_k):
    f = workloads.bi_maxwellian(33, 3, 8, 8.0, seed=12)
    Q = _gpu_collide(bz, 3, 8, 8.0, 1.0, f, "fp32")
    fin = as_input(f, "fp32")
    k = oracle_k(3, 8, 8.0, 1.0)
    Qr = k.collide(fin)
    assert relerr(Q, Qr) < TOL32
    check_fp32_cells(k, fin, Q, Qr, what="fp32 3-D 8^3")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_sizes(bz, oracle_k, precision):
    import torch
    # one cell, the smallest grid (h = 1)
    f = workloads.bi_maxwellian(1, 2, 4, 3.0, seed=3)
    Q = _gpu_collide(bz, 2, 4, 3.0, 1.0, f, precision)
    Qr = oracle_k(2, 4, 3.0, 1.0).collide(as_input(f, precision))
    assert relerr(Q, Qr) < (TOL64 if precision == "fp64" else TOL32)
    # zero cells: a no-op that leaves Q untouched
    m = bz.Modes(bz.Grid(2, 16, 8.0), 1.0)
    dt = torch.float64 if precision == "fp64" else torch.float32
    f0 = torch.zeros((0, 256), dtype=dt, device="cuda")
    Q0 = torch.zeros((0, 256), dtype=dt, device="cuda")
    bz.collide_batch(m, f0, Q0, precision=precision)
    bz.check()


def test_largest_grid_fp64(bz, oracle_k):
    """N = 64 (the largest 2-D grid the library accepts), a ragged 3 cells."""
    f = workloads.bi_maxwellian(3, 2, 64, 12.0, seed=4)
    Q = _gpu_collide(bz, 2, 64, 12.0, 0.0, f, "fp64")
    Qr = oracle_k(2, 64, 12.0, 0.0).collide(f)
    assert relerr(Q, Qr) < TOL64


def test_argument_errors(bz):
    import torch
    m = bz.Modes(bz.Grid(2, 16, 8.0), 1.0)
    f = torch.zeros((4, 256), dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):
        bz.collide_batch(m, f, precision="fp64")
    with pytest.raises(bz.BzError) as e:
        bz.collide_batch(m, f, f, precision="fp32")          # f and Q overlap
    assert e.value.code == bz.EINVAL
    lib = bz.load()
    assert lib.collide_batch(m._h, 7, 0, f.data_ptr(), f.data_ptr() + 1, 4, None) == bz.EINVAL


def test_check_input_flags_nonfinite(bz):
    import torch
    m = bz.Modes(bz.Grid(2, 16, 8.0), 1.0)
    f = torch.ones((5, 256), dtype=torch.float32, device="cuda")
    f[3, 17] = float("nan")
    bz.collide_batch(m, f, precision="fp32", check_input=True)
    with pytest.raises(bz.BzError) as e:
        bz.check()
    assert e.value.code == bz.ENONFINITE
    bz.check()                                  # the error word was cleared
    f[3, 17] = 1.0
    bz.collide_batch(m, f, precision="fp32", check_input=True)
    bz.check()


@pytest.mark.parametrize("precision,N", [("fp64", 32), ("fp32", 32), ("fp32", 48), ("fp32", 24)])
def test_deterministic_and_mass_conserving(bz, precision, N):
    f = workloads.bi_maxwellian(50, 2, N, 10.0, seed=8, noise=0.05)
    m = bz.Modes(bz.Grid(2, N, 10.0), 1.0)
    x = to_dev(f, precision)
    Q1 = bz.collide_batch(m, x, precision=precision).cpu().numpy()
    Q2 = bz.collide_batch(m, x, precision=precision).cpu().numpy()
    assert np.array_equal(Q1, Q2)
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert np.abs(Q1.sum(axis=1)).max() < tol * np.abs(Q1).sum(axis=1).max()


def test_full_size_fp32_sampled(bz, oracle_k):
    """65536 cells, 32^2, VHS, shifted Maxwellians (Mach 0-3): the launch the
    benchmark times.  4096 sampled cells (every 16th, and both ends of the
    batch) against the oracle at the 1e-6 target; 256 of them also against
    the per-cell bounds."""
    n = 65536
    f = workloads.shifted_maxwellians(n, 2, 32, 10.0, seed=1003).astype(np.float32)
    Q = _gpu_collide(bz, 2, 32, 10.0, 1.0, f, "fp32")
    assert np.isfinite(Q).all()
    idx = np.unique(np.concatenate([np.arange(0, n, 16), [1, 31, 32, 65503, 65535]]))
    k = oracle_k(2, 32, 10.0, 1.0)
    Qr = k.collide(f[idx].astype(np.float64))
    err = relerr(Q[idx], Qr)
    print("full-size fp32 rel-L2 over %d cells: %.3e" % (len(idx), err))
    assert err < TARGET32
    sub = np.arange(0, len(idx), len(idx) // 256)
    check_fp32_cells(k, f[idx[sub]].astype(np.float64), Q[idx[sub]], Qr[sub], what="full-size fp32")


def test_full_size_fp64_every_cell(bz, oracle_k):
    """4096 cells, 32^2, VHS, bi-Maxwellian with 5% noise (plain form): every
    cell against the oracle, element by element."""
    n = 4096
    f = workloads.bi_maxwellian(n, 2, 32, 10.0, seed=1002, noise=0.05)
    Q = _gpu_collide(bz, 2, 32, 10.0, 1.0, f, "fp64")
    Qr = oracle_k(2, 32, 10.0, 1.0).collide(f)
    assert relerr(Q, Qr) < TOL64
    cellmax = np.abs(Qr).max(axis=1, keepdims=True)
    worst = (np.abs(Q - Qr) / cellmax).max()
    print("fp64 config 2: rel-L2 %.3e, worst element / cell max %.3e" % (relerr(Q, Qr), worst))
    assert worst < TOL64
