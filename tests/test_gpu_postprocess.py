"""Post-processing of T(E) on the GPU: the Landauer current (Eq. Landauer)
against the oracle's trapezoidal integral of the same T, and on the waveguide
against the area under its open-channel staircase; the insensitivity of T(E)
to the Gaussian absorbing potential's height and width (Eq. ABC; Sec. III
reports robustness to 100% changes of the height and ~23% of the width)."""
import numpy as np
import pytest

import oracle as O
from paper_1401_0782_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0782_gb300 import binding
    return binding


def test_landauer_kernel_matches_oracle(B):
    ctx = B.Context(0)
    rng = np.random.default_rng(3)
    E = np.sort(rng.uniform(-1.0, 2.0, 3001))
    T = np.abs(rng.standard_normal(E.size))
    V = np.array([-0.7, -0.1, 0.0, 0.05, 0.3, 1.2])
    for E_F, kT in ((0.2, 0.0), (0.5, 0.01), (1.0, 0.1)):
        I = ctx.landauer_current(E, T, V, E_F, kT)
        I_ref = O.landauer_current(E, T, V, E_F, kT)
        assert np.allclose(I, I_ref, rtol=1e-12, atol=1e-15), (E_F, kT, I, I_ref)
    with pytest.raises(B.RsnError) as e:
        ctx.landauer_current(E[::-1], T, V)
    assert e.value.code == B.RSN_EINVAL
    with pytest.raises(B.RsnError) as e:
        ctx.landauer_current(E, T, V, kT=-1.0)
    assert e.value.code == B.RSN_EINVAL
    ctx.close()


def test_waveguide_current_from_shifted_transmission(B):
    w = P.waveguide()
    ctx = B.Context(0).set_junction(w)
    E = np.linspace(0.3, 2.0, 171)
    T = ctx.transmission_shifted(E, None, B.default_opts(B.RSN_FP64))
    E_F, V = 0.85, np.array([0.2, 0.3, -0.3])
    I = ctx.landauer_current(E, T, V, E_F)
    assert np.allclose(I, O.landauer_current(E, T, V, E_F), rtol=1e-12, atol=1e-15)
    # the bias windows [0.70, 1.00] Ha lie between the first two thresholds
    # (0.4825 and 1.1771 Ha), at least 0.17 Ha from either, where one channel
    # is open and the CAP staircase holds to 0.06: I = V / pi there
    for v, i in zip(V, I):
        assert abs(i - v / np.pi) <= 0.06 * abs(v) / np.pi, (v, i, v / np.pi)
    ctx.close()


def test_abc_insensitivity_scan(B):
    # Gaussian ABCs centred on the end planes (Eq. ABC), height doubled and
    # width raised by 23% about a working point: T(E) stays on the staircase
    # away from the thresholds, and the three scans agree
    E = np.array([0.3, 0.75, 0.95, 1.45, 1.65])
    n_open = np.array([O.open_channels(8, 8, 0.5, e) for e in E])
    scans = []
    for g0, sg in ((0.5, 4.0), (1.0, 4.0), (0.5, 4.9)):
        w = P.waveguide(cap="gaussian", gamma0=g0, sigma=sg)
        ctx = B.Context(0).set_junction(w)
        T = ctx.transmission_shifted(E, None, B.default_opts(B.RSN_FP64))
        assert np.allclose(T, O.transmission(w, E), rtol=1e-9, atol=1e-12)
        scans.append(T)
        ctx.close()
    scans = np.array(scans)
    assert np.abs(scans - n_open[None, :]).max() <= 0.1, (scans, n_open)
    assert np.abs(scans - scans[0][None, :]).max() <= 0.1
