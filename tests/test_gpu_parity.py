"""GPU path (through the C-ABI) against the FP64 CPU oracle, stage by stage.

Bars: tree, leaf assignment and interaction lists bit-exact (as sets);
FP64 path within 1e-12 relative RMS of the oracle; mixed path within 1e-5
(FP32 bulk with FP64 derivative tensors and FP64 local accumulation).  The
relative RMS is sqrt(sum |H - H_ref|^2 / sum |H_ref|^2) over the compared
dipoles.  The mixed path is also held to the local bounds of
``local_parity``: every dipole's field error and every cell's Taylor
coefficients against the oracle's.  Inputs are the seeded workloads of
``paper_0810_0233_gb300.workloads``.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import workloads as W

import local_parity as LP

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-5


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def run_gpu(pos, mom, p, theta, leaf=0.0, box=None, prec="fp64"):
    with C.FMM(pos, mom, p, theta, leaf, box=box, precision=prec) as f:
        H, E = f.field_energy()
        st = f.stats()
        extra = dict(axes=f.axes(), leaf_of=f.leaf_of(), near=f.pairs("near"), far=f.pairs("far"),
                     Q=f.expansions("Q"), V=f.expansions("V"))
    return H, E, st, extra


def nonempty_cells(leaf_of, L):
    """Set of heap ids of non-empty cells at every level."""
    ne = set()
    for l in range(L + 1):
        for k in np.unique(leaf_of >> (L - l)):
            ne.add((1 << l) + int(k))
    return ne


def oracle_pairs(f, ne, kind):
    pr = f.near_pairs() if kind == "near" else f.far_pairs()
    return {(int(a), int(b)) for a, b in pr if int(a) in ne and int(b) in ne}


def lib_to_oracle_cols(p):
    mi = C.multi_indices(p)
    return np.array([O.index(n) for n in mi])


def check_full(pos, mom, p, theta, leaf=0.0, box=None, lists=True, expansions=True):
    Href, Eref, f = O.fmm_field(pos, mom, p, theta, leaf, box=box)
    H, E, st, ex = run_gpu(pos, mom, p, theta, leaf, box, "fp64")
    L = f.depth
    assert st["depth"] == L
    assert list(ex["axes"]) == list(f.axes())
    assert np.array_equal(ex["leaf_of"], f.leaf_of())
    if lists:
        ne = nonempty_cells(f.leaf_of(), L)
        assert {tuple(map(int, x)) for x in ex["near"]} == oracle_pairs(f, ne, "near")
        assert {tuple(map(int, x)) for x in ex["far"]} == oracle_pairs(f, ne, "far")
    if expansions:
        perm = lib_to_oracle_cols(p)
        Qo = f.moments()[:, perm]
        Vo = f.locals()[:, perm]
        ne = sorted(nonempty_cells(f.leaf_of(), L))
        assert rel(ex["Q"][ne], Qo[ne]) < TOL64
        if np.abs(Vo[ne]).max() > 0:
            for l in range(2, L + 1):
                rows = [c for c in ne if (c >> l) == 1]
                if np.abs(Vo[rows]).max() > 0:
                    assert rel(ex["V"][rows], Vo[rows]) < TOL64, l
    assert rel(H, Href) < TOL64
    assert abs(E - Eref) <= TOL64 * abs(Eref) + 1e-300
    Hm, Em, stm, exm = run_gpu(pos, mom, p, theta, leaf, box, "mixed")
    assert rel(Hm, Href) < TOLMIX
    assert abs(Em - Eref) <= 10 * TOLMIX * abs(Eref)
    check_local(Hm, Href, exm["V"], f)
    return Href, H, Hm, st


def check_local(Hm, Href, Vm, f):
    """Mixed path, local bounds: every dipole, and every non-empty cell of
    levels >= 2 (the levels that receive far interactions) against the
    oracle's Taylor coefficients."""
    assert LP.dipole_max_err(Hm, Href) < LP.DIPOLE_TOL
    L = f.depth
    Vo = f.locals()[:, lib_to_oracle_cols(f.p)]
    cells = [c for c in nonempty_cells(f.leaf_of(), L) if c >= 4]
    if cells and np.abs(Vo[cells]).max() > 0:
        err = LP.cell_errors(Vm, Vo, cells, C.multi_indices(f.p), f.box(), f.axes())
        assert max(err.values()) < LP.CELL_TOL, err


# ---------------------------------------------------------------- workloads

def test_c1_lattice_p4():
    """10^3 simple-cubic lattice, p = 4, theta = 0.5, s = 8, lattice-cell box."""
    pos, mom, box = W.lattice(10)
    Href, H, Hm, st = check_full(pos, mom, 4, 0.5, 8.0, box)
    assert st["depth"] == 7 and st["far_pairs"] == 4008
    Hd = O.direct_field(pos, mom)
    assert rel(H, Hd) < 1e-3


def test_ferrofluid_p6_several_tiles():
    """20k ferrofluid points (same density as the 10^6 workload), p = 6,
    theta = 0.5, Eq. so leaves: several M2L tiles per level and ragged
    near-field batches."""
    pos, mom = W.ferrofluid(20000, side=100.0 * (0.02) ** (1 / 3), seed=W.BASE_SEED + 12)
    Href, H, Hm, st = check_full(pos, mom, 6, 0.5)
    assert st["depth"] >= 9
    sub = W.subset(len(pos), 500, 1)
    Hd = O.direct_field(pos, mom, targets=sub)
    assert rel(Hm[sub], Hd) < 1e-4


def test_ring_p6_theta04():
    """Thin-film ring (scaled down), vortex moments, p = 6, theta = 0.4."""
    pos, mom = W.ring(r_out=48.0, r_in=16.0, seed=W.BASE_SEED + 13)
    check_full(pos, mom, 6, 0.4)


def test_clustered_empty_leaves():
    pos, mom = W.clustered(6000, seed=W.BASE_SEED + 14)
    Href, H, Hm, st = check_full(pos, mom, 5, 0.5)
    assert st["nonempty_leaves"] < 2 ** st["depth"]


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_every_order(p):
    rng = np.random.default_rng(100 + p)
    pos = rng.uniform(0, 14, size=(2500, 3))
    mom = W.unit_vectors(2500, rng)
    check_full(pos, mom, p, 0.5, 6.0, expansions=(p in (1, 6, 8)))


@pytest.mark.parametrize("theta", [0.25, 0.7, 0.95])
def test_theta_range(theta):
    rng = np.random.default_rng(7)
    pos = rng.uniform(0, 12, size=(3000, 3))
    mom = W.unit_vectors(3000, rng)
    check_full(pos, mom, 4, theta, 8.0, expansions=False)


# ---------------------------------------------------------------- edge cases

def test_single_dipole():
    H, E, st, _ = run_gpu(np.array([[1.0, 2.0, 3.0]]), np.array([[0.0, 0.0, 1.0]]), 4, 0.5)
    assert np.all(H == 0) and E == 0.0 and st["depth"] == 0


def test_two_dipoles_and_single_leaf():
    pos = np.array([[0.0, 0, 0], [1.5, 0, 0]])
    mom = np.array([[1.0, 0, 0], [1.0, 0, 0]])
    H, E, st, _ = run_gpu(pos, mom, 3, 0.5)
    assert np.allclose(H[1], [2 / 1.5**3, 0, 0], rtol=1e-14)
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 5, size=(300, 3))
    mom = W.unit_vectors(300, rng)
    H, E, st, _ = run_gpu(pos, mom, 4, 0.5, leaf=1000.0)
    assert st["depth"] == 0
    assert rel(H, O.direct_field(pos, mom)) < TOL64


def test_coincident_points_skipped():
    rng = np.random.default_rng(4)
    pos = rng.uniform(0, 6, size=(800, 3))
    pos[10] = pos[11]
    mom = W.unit_vectors(800, rng)
    check_full(pos, mom, 4, 0.5, 8.0, expansions=False)


def test_flat_and_box_boundary():
    """A single lattice plane (flat tree), and a box whose faces carry points."""
    pos, mom, box = W.lattice(24, 24, 1, seed=W.BASE_SEED + 15)
    check_full(pos, mom, 4, 0.5, 8.0, box=box)
    pos, mom, _ = W.lattice(9, 7, 5, seed=W.BASE_SEED + 16)
    box = np.array([0.0, 0.0, 0.0, 8.0, 6.0, 4.0])
    check_full(pos, mom, 3, 0.6, 4.0, box=box, expansions=False)


def test_device_and_host_pointers_agree_and_repeat():
    torch = pytest.importorskip("torch")
    pos, mom = W.ferrofluid(5000, side=100.0 * 0.005 ** (1 / 3), seed=W.BASE_SEED + 17)
    with C.FMM(pos, mom, 5, 0.5) as f:
        H1 = f.field()
        H2 = f.field()
    dp = torch.from_numpy(pos).cuda()
    dm = torch.from_numpy(mom).cuda()
    with C.FMM(dp, dm, 5, 0.5, stream=torch.cuda.current_stream()) as f:
        Hd = torch.zeros((len(pos), 3), dtype=torch.float64, device="cuda")
        f.field(Hd)
        torch.cuda.synchronize()
    assert np.array_equal(H1, H2)
    assert np.array_equal(H1, Hd.cpu().numpy())


def test_set_moments_and_set_positions():
    rng = np.random.default_rng(8)
    pos = rng.uniform(0, 10, size=(3000, 3))
    mom = W.unit_vectors(3000, rng)
    mom2 = W.unit_vectors(3000, rng)
    pos2 = rng.uniform(0, 10, size=(3000, 3))
    with C.FMM(pos, mom, 4, 0.5, precision="fp64") as f:
        f.field()
        f.set_moments(mom2)
        Ha = f.field()
        f.set_positions(pos2, mom)
        Hb = f.field()
    assert rel(Ha, O.fmm_field(pos, mom2, 4, 0.5)[0]) < TOL64
    assert rel(Hb, O.fmm_field(pos2, mom, 4, 0.5)[0]) < TOL64


def test_direct_kernel_matches_oracle():
    rng = np.random.default_rng(9)
    pos = rng.uniform(0, 10, size=(3000, 3))
    mom = W.unit_vectors(3000, rng)
    t = W.subset(3000, 300, 2)
    assert rel(C.direct_field(pos, mom, targets=t), O.direct_field(pos, mom, targets=t)) < 1e-14
    assert rel(C.direct_field(pos, mom), O.direct_field(pos, mom)) < 1e-14


# ---------------------------------------------------------------- errors

def test_invalid_arguments_rejected():
    pos = np.zeros((4, 3))
    pos[:, 0] = np.arange(4)
    mom = np.ones((4, 3))
    for kw in (dict(p=0), dict(p=9), dict(theta=0.0), dict(theta=1.0), dict(leaf_size=0.5)):
        args = dict(p=4, theta=0.5, leaf_size=0.0)
        args.update(kw)
        with pytest.raises(C.CCFMMError) as e:
            C.FMM(pos, mom, args["p"], args["theta"], args["leaf_size"])
        assert e.value.status == C.ERR_ARG
    bad = pos.copy()
    bad[2, 1] = np.nan
    with pytest.raises(C.CCFMMError) as e:
        C.FMM(bad, mom, 4, 0.5)
    assert e.value.status == C.ERR_ARG and "non-finite" in str(e.value)
    badm = mom.copy()
    badm[1, 2] = np.inf
    with pytest.raises(C.CCFMMError):
        C.FMM(pos, badm, 4, 0.5)
    with pytest.raises(C.CCFMMError) as e:
        C.FMM(pos, mom, 4, 0.5, box=[0, 0, 0, 2, 1, 1])
    assert "outside" in str(e.value)
    # the context stays usable after rejected calls
    with C.FMM(pos, mom, 4, 0.5) as f:
        assert np.all(np.isfinite(f.field()))


def test_injected_allocation_failure():
    """CCFMM_FAIL_ALLOC=k fails the k-th device allocation: the call returns
    CCFMM_ERR_ALLOC, nothing leaks into a crash, and a later call works."""
    code = (
        "import numpy as np, sys\n"
        "sys.path.insert(0, %r)\n"
        "from paper_0810_0233_gb300 import ccfmm as C\n"
        "pos = np.random.default_rng(0).uniform(0, 5, (500, 3)); mom = np.ones((500, 3))\n"
        "try:\n"
        "    C.FMM(pos, mom, 4, 0.5)\n"
        "    print('NOFAIL')\n"
        "except C.CCFMMError as e:\n"
        "    print('STATUS', e.status)\n"
        "f = C.FMM(pos, mom, 4, 0.5); H = f.field(); f.close()\n"
        "print('AFTER', bool(np.isfinite(H).all()))\n" % os.path.dirname(os.path.dirname(
            os.path.abspath(__file__))))
    env = dict(os.environ, CCFMM_FAIL_ALLOC="5")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert "STATUS -2" in r.stdout and "AFTER True" in r.stdout, r.stdout


def test_near_pair_count_from_the_lists():
    """fmm_stats' p2p_pairs (counted on demand once per build) equals the
    ordered near pairs i != j implied by the leaf near lists, before and
    after a rebuild."""
    pos, mom = W.ferrofluid(20000, side=100.0 * 0.02 ** (1 / 3), seed=W.BASE_SEED + 61)
    with C.FMM(pos, mom, 6, 0.5) as f:
        for step in range(2):
            if step:
                pos = pos * 0.7
                f.set_positions(pos, mom)
            st = f.stats()
            L = st["depth"]
            cnt = np.bincount(f.leaf_of(), minlength=1 << L)
            pr = f.pairs("near") - (1 << L)
            assert st["p2p_pairs"] == int((cnt[pr[:, 0]] * cnt[pr[:, 1]]).sum()) - len(pos)


@pytest.mark.parametrize("kind", ["ferrofluid", "clustered", "lattice"])
@pytest.mark.parametrize("overlap", ["1", "0"])
@pytest.mark.parametrize("mode", ["sym"])
def test_near_field_variants(monkeypatch, kind, overlap, mode):
    """The symmetric near field (CCFMM_P2P=sym: each pair of near leaves
    once, both directions, Newton's third law; unordered global reductions)
    against the oracle and the default one-sided kernel: the same sums in
    another order, so FP32 rounding apart they agree."""
    if kind == "ferrofluid":
        pos, mom = W.ferrofluid(20000, side=100.0 * 0.02 ** (1 / 3), seed=W.BASE_SEED + 18)
        box = None
    elif kind == "clustered":
        pos, mom = W.clustered(12000, seed=W.BASE_SEED + 19)
        box = None
    else:
        pos, mom, box = W.lattice(17, 13, 11, seed=W.BASE_SEED + 20)
    monkeypatch.setenv("CCFMM_OVERLAP", overlap)
    Href, Eref, f = O.fmm_field(pos, mom, 6, 0.5, box=box)
    monkeypatch.delenv("CCFMM_P2P", raising=False)
    H0, E0, _, _ = run_gpu(pos, mom, 6, 0.5, box=box, prec="mixed")
    monkeypatch.setenv("CCFMM_P2P", mode)
    H1, E1, st, ex = run_gpu(pos, mom, 6, 0.5, box=box, prec="mixed")
    assert rel(H1, Href) < TOLMIX
    assert abs(E1 - Eref) <= 10 * TOLMIX * abs(Eref)
    check_local(H1, Href, ex["V"], f)
    assert rel(H1, H0) < 2e-6

