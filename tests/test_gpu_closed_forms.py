"""Pure-absorber closed forms through the library's own precision forms.

With no scattering and each absorption ending its package (dies_run_frozen
with DIES_FROZEN_ABSORB_TERMINAL | DIES_FROZEN_FORM), the expected energy a
shell absorbs is fixed by the geometry alone (Sect. 2.1, Eq. 4): an
impact-parameter quadrature for the isotropic external field and the radial
attenuation for the central source.  At 1e8 packages this resolves the
absorbed fraction of well-filled shells to ~1e-4, so it checks the FP32
stepping of the MIXED and FP32 forms (compensated R_b^2 - p^2, the hardware
reciprocal square root, one column density per flight, forced first
interaction) far below the 1 % temperature gate, which the FP64 form's
bit-exact frozen pass cannot do (it runs different code).

Each package deposits its whole energy (weight <= 1 with forcing) in at most
one shell, so the count variance N P (1 - P) bounds the variance of E/eps."""
import numpy as np
import pytest

import closed_forms as CF
from gpu_util import check_against_expectation
from paper_2408_13807_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_13807_gb300 import build as B
    B.build()
    from paper_2408_13807_gb300 import dies
    dies.load()
    return dies


def _source_fractions(oracle, cloud):
    S = (cloud.J_ext if cloud.J_ext is not None else cloud.point_spec) * oracle.freq_weights(cloud.freq)
    return S / S.sum()


def _pure_absorber(cloud):
    return cloud.replace(ksca=np.zeros_like(cloud.ksca))


def _grey_log(n, r_in, tau, external, ffi=0):
    """Grey pure absorber on log-spaced shells r_in..1 (inner void): BE-like
    density for the external field, r^-2 around the point source."""
    radii = W.log_radii(n, r_in)
    shape = W.be_like(radii, 0.1) if external else W.power_law(radii, -2.0)
    m = W.grey_model(n, tau, external=external, L_point=0.0 if external else W.L_SUN)
    rho = shape / np.sum(shape * np.diff(radii))  # radial column 1: tau = kabs * 1 = tau
    return m.replace(radii=radii, rho=rho, ffi=int(ffi))


def _expected(oracle, cloud):
    """Absorbed fraction per shell, summed over the source spectrum, and
    the escaping fraction per frequency bin."""
    p = _source_fractions(oracle, cloud)
    K = cloud.kabs[:, None] * cloud.rho[None, :]
    use = p > 0
    f = np.zeros((cloud.n_freq, cloud.n_cells))
    if cloud.J_ext is not None:
        f[use] = CF.external_shell_absorption_annuli(cloud.radii, K[use])
    else:
        for k in np.nonzero(use)[0]:
            f[k] = CF.point_shell_absorption(cloud.radii, K[k])
    return (p[:, None] * f).sum(0), p * (1.0 - f.sum(1))


CASES = {
    # 128 equal shells, the benchmark dust law without scattering, 64 bins
    "c2_AV1": lambda: _pure_absorber(W.external_cloud(128, 1.0)),
    "c2_AV10": lambda: _pure_absorber(W.external_cloud(128, 10.0)),
    # 1024 log shells 1e-6..1 (grey): external field plain and forced, point source
    "c5_ext_grey": lambda: _grey_log(1024, 1e-6, 2.0, True),
    "c5_ext_grey_ffi": lambda: _grey_log(1024, 1e-6, 0.1, True, ffi=1),
    "c5_pt_grey": lambda: _grey_log(1024, 1e-6, 5.0, False),
}
FORMS = [("mixed", 0.0), ("mixed", 1e-2), ("fp32", 0.0)]


@pytest.fixture(scope="module")
def expectations(oracle):
    return {name: _expected(oracle, make()) for name, make in CASES.items()}


@pytest.mark.parametrize("form", FORMS, ids=["mixed", "mixed_fp64_inner", "fp32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_pure_absorber_shells_in_the_precision_forms(D, expectations, name, form):
    cloud = CASES[name]()
    prec, r64 = form
    N = 100_000_000
    m = D.Model(cloud, precision=prec, fp64_radius=r64)
    m.run_terminal_in_form(N, seed=23)
    st = m.stats()
    assert st["status_word"] == 0 and st["injected"] == N
    L = st["E_injected"]
    E, sed = m.absorbed(), m.sed()
    # (escaping weights are tallied in units of 2^-24 package energies)
    assert E.sum() + sed.sum() + st["E_lost"] == pytest.approx(L, rel=1e-6)
    P, esc = expectations[name]
    # absorbed energy per shell in package units against N P, variance <= N P (1 - P)
    z = check_against_expectation(E / L * N, N * P, N * P * (1.0 - P), min_expect=400.0)
    # escaping energy per frequency bin
    check_against_expectation(sed / L * N, N * esc, N * esc * (1.0 - esc), min_expect=400.0)
    filled = int(np.sum(N * P > 400.0))
    assert filled >= (20 if name.startswith("c5") else 100), filled
    m.close()
    print(f"{name} {prec} fp64_radius={r64}: {filled} shells, max |z| {np.abs(z).max():.2f}")


def test_terminal_form_pass_rejects_records(D):
    cloud = CASES["c2_AV1"]()
    m = D.Model(cloud, precision="mixed")
    with pytest.raises(D.DiesError) as ei:
        D.dies_run_frozen(m.h, np.full(cloud.n_cells, 10.0), 10, 1,
                          D.DIES_FROZEN_ABSORB_TERMINAL | D.DIES_FROZEN_FORM, 10, True)
    assert ei.value.code == D.DIES_EINVAL
    with pytest.raises(D.DiesError):
        D.dies_run_frozen(m.h, np.full(cloud.n_cells, 10.0), 10, 1, D.DIES_FROZEN_FORM, 0, False)
    m.close()
