"""The CUDA spectra (efe_absorption_spectrum, efe_power_spectrum) against the
oracle's on the same traces."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _traces(n_t, dt, seed=3):
    """Three kicked runs: a sum of damped oscillators per axis plus cross terms."""
    rng = np.random.default_rng(seed)
    t = dt * np.arange(n_t)
    mu = np.zeros((3, n_t, 3))
    for j in range(3):
        for k in range(3):
            for _ in range(4):
                w0, f, g = rng.uniform(0.2, 2.5), rng.uniform(0.1, 1.0), rng.uniform(0.005, 0.05)
                mu[j, :, k] += 1e-3 * f / w0 * np.sin(w0 * t) * np.exp(-0.5 * g * t)
            mu[j, :, k] += rng.normal()   # static dipole
    return mu


@pytest.mark.parametrize("n_t,n_om", [(2001, 257), (3, 5), (10000, 1000)])
def test_absorption_matches_oracle(n_t, n_om):
    from oracle import spectra
    from paper_2210_14421_gb300 import absorption_spectrum
    dt, tau, kappa = 0.05, 100.0, 2e-3
    mu = _traces(n_t, dt)
    om = np.linspace(0.01, 3.0, n_om)
    ref = spectra.absorption_spectrum(mu, dt, om, tau, kick=kappa)
    got = absorption_spectrum(_dev(mu), dt, _dev(om), tau, kick=kappa).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-10 * max(np.max(np.abs(ref)), 1e-300)
    # the same with the perturbing field given by samples (a Gaussian pulse)
    t = dt * np.arange(n_t)
    E = kappa * np.exp(-(t - 1.0) ** 2 / (2 * 0.2 ** 2))
    ref2 = spectra.absorption_spectrum(mu, dt, om, tau, field=E)
    got2 = absorption_spectrum(_dev(mu), dt, _dev(om), tau, field=_dev(E)).cpu().numpy()
    assert np.max(np.abs(got2 - ref2)) <= 1e-10 * max(np.max(np.abs(ref2)), 1e-300)


def test_absorption_with_strided_traces():
    """Traces stored sample-major ([n][j][k], as a batch of three polarisations
    is recorded step by step) give the same spectrum."""
    from paper_2210_14421_gb300 import absorption_spectrum
    dt, tau, kappa = 0.05, 100.0, 1e-3
    mu = _traces(1500, dt, seed=5)
    om = _dev(np.linspace(0.05, 2.0, 64))
    a = absorption_spectrum(_dev(mu), dt, om, tau, kick=kappa)
    sm = _dev(np.transpose(mu, (1, 0, 2))).permute(1, 0, 2)   # strides (3, 9, 1)
    b = absorption_spectrum(sm, dt, om, tau, kick=kappa)
    assert torch.equal(a, b)


@pytest.mark.parametrize("n_t,n_om", [(4001, 513), (3, 2)])
def test_power_spectrum_matches_oracle(n_t, n_om):
    from oracle import spectra
    from paper_2210_14421_gb300 import power_spectrum
    dt, tau = 0.1, 1e5
    t = dt * np.arange(n_t)
    mu = 0.3 * np.sin(0.057 * t) + 0.01 * np.sin(3 * 0.057 * t) + 1e-3 * np.sin(5 * 0.057 * t + 0.3)
    om = np.linspace(0.0, 0.4, n_om)
    ref = spectra.power_spectrum(mu, dt, om, tau)
    got = power_spectrum(_dev(mu), dt, _dev(om), tau).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-10 * max(np.max(np.abs(ref)), 1e-300)


def test_spectra_at_size_on_sampled_frequencies():
    """100,001 samples x 4,096 frequencies on the device; 48 of the frequencies
    checked against the oracle one by one."""
    from oracle import spectra
    from paper_2210_14421_gb300 import absorption_spectrum, power_spectrum
    dt, tau, kappa = 0.02, 100.0, 1e-3
    n_t = 100001
    mu = _traces(n_t, dt, seed=9)
    om = np.linspace(0.001, 4.0, 4096)
    S = absorption_spectrum(_dev(mu), dt, _dev(om), tau, kick=kappa).cpu().numpy()
    P = power_spectrum(_dev(mu[0, :, 0]), dt, _dev(om), 1e4).cpu().numpy()
    idx = np.random.default_rng(1).choice(len(om), 48, replace=False)
    Sr = spectra.absorption_spectrum(mu, dt, om[idx], tau, kick=kappa)
    Pr = spectra.power_spectrum(mu[0, :, 0], dt, om[idx], 1e4)
    assert np.max(np.abs(S[idx] - Sr)) <= 1e-9 * np.max(np.abs(Sr))
    assert np.max(np.abs(P[idx] - Pr)) <= 1e-9 * np.max(np.abs(Pr))


def test_spectra_reject_bad_arguments():
    from paper_2210_14421_gb300 import EfeError, absorption_spectrum, power_spectrum
    mu = torch.zeros((3, 10, 3), dtype=torch.float64, device="cuda")
    om = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(EfeError):
        absorption_spectrum(mu, 0.0, om, 1.0, kick=1.0)
    with pytest.raises(EfeError):
        absorption_spectrum(mu, 0.1, om, 1.0)              # neither field nor kick
    with pytest.raises(EfeError):
        power_spectrum(mu[0, :2, 0], 0.1, om, 1.0)           # fewer than three samples
