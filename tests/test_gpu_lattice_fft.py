"""The lattice FFT comparator (fmm_lattice_*, Sec. V) against the oracle's
O(N^2) direct sum: the zero-padded convolution is the open-boundary sum of
Eq. H2 exactly, so the FP64 transforms must agree with the direct sum to
rounding, the FP32 ones to single precision; on the paper's lattice
benchmark both methods (FFT and the fast multipole method) must agree."""
import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import workloads as W

import local_parity as LP

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.mark.parametrize("dims,spacing", [((10, 10, 10), 1.0), ((7, 5, 3), 0.7),
                                          ((16, 16, 1), 1.0), ((9, 1, 1), 2.0),
                                          ((1, 6, 4), 1.0)])
def test_fft_equals_direct_sum(dims, spacing):
    pos, mom, _ = W.lattice(*dims, spacing=spacing, seed=W.BASE_SEED + 70)
    Hd = O.direct_field(pos, mom)
    Ed = O.energy_from_field(mom, Hd)
    with C.Lattice(*dims, spacing=spacing, precision="fp64") as lat:
        H, E = lat.field_energy(mom)
    assert rel(H, Hd) < 1e-12
    assert abs(E - Ed) <= 1e-12 * abs(Ed)
    with C.Lattice(*dims, spacing=spacing, precision="mixed") as lat:
        H32, E32 = lat.field_energy(mom)
    assert rel(H32, Hd) < 1e-5
    assert LP.dipole_max_err(H32, Hd) < LP.DIPOLE_TOL
    assert abs(E32 - Ed) <= 1e-5 * abs(Ed)


def test_single_site_and_device_buffers():
    torch = pytest.importorskip("torch")
    with C.Lattice(1, 1, 1) as lat:
        H, E = lat.field_energy(np.array([[0.0, 0.0, 1.0]]))
    assert np.all(H == 0) and E == 0.0
    pos, mom, _ = W.lattice(8, 6, 5, seed=W.BASE_SEED + 71)
    with C.Lattice(8, 6, 5) as lat:
        Hh, Eh = lat.field_energy(mom)
        md = torch.from_numpy(mom).cuda()
        Hdv = torch.zeros((len(mom), 3), dtype=torch.float64, device="cuda")
        _, Ed = lat.field_energy(md, out=Hdv)
        Hh2, _ = lat.field_energy(mom)
    assert np.array_equal(Hdv.cpu().numpy(), Hh) and Ed == Eh
    assert np.array_equal(Hh2, Hh)


def test_fft_and_fmm_agree_on_the_lattice_benchmark():
    """The paper's benchmark (a 32^3 simple-cubic lattice of random unit
    dipoles, Sec. IV) by both methods: the FFT result is exact, so the FMM's
    error against it is the FMM's truncation error."""
    pos, mom, box = W.lattice(32, seed=W.BASE_SEED + 72)
    with C.Lattice(32, precision="fp64") as lat:
        Hf, Ef = lat.field_energy(mom)
    sub = W.subset(len(pos), 400, 8)
    assert rel(Hf[sub], O.direct_field(pos, mom, targets=sub)) < 1e-12
    with C.FMM(pos, mom, 6, 0.5, box=box, precision="mixed") as f:
        Hm, Em = f.field_energy()
    assert rel(Hm, Hf) < 1e-4
    assert abs(Em - Ef) < 1e-4 * abs(Ef)


def test_rejects_bad_arguments():
    for args in ((0, 4, 4), (4, -1, 4), (5000, 2, 2)):
        with pytest.raises(C.CCFMMError) as e:
            C.Lattice(*args)
        assert e.value.status == C.ERR_ARG
    with pytest.raises(C.CCFMMError):
        C.Lattice(4, spacing=0.0)
    with pytest.raises(C.CCFMMError):
        C.Lattice(4, precision="fp64").field_energy(np.full((64, 3), np.nan))
