"""The CUDA adjoint (efe_adjoint_dipole) against the oracle's exact discrete
adjoint and against central finite differences of the CUDA forward run."""
import dataclasses

import numpy as np
import pytest

import efe_workloads as W

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


# (workload, field, dt, n_steps, window, direction)
CASES = {
    "one_atom_p2_sine_gauss": (
        lambda: W.small_cluster(n_atoms=1, cells_per_axis=3, degree=2, n_quad=4, L=10.0, n_orb=1, Zval=2.0),
        W.Field(kind=W.FIELD_SINE_GAUSS, amp=0.05, omega=0.8, t0=0.2, sigma=0.3, direction=(1.0, 0.0, 0.0)),
        0.05, 6, (4, 6), (1.0, 0.0, 0.0)),
    "two_atoms_p3_gauss": (
        lambda: W.small_cluster(n_atoms=2, cells_per_axis=3, degree=3, n_quad=5, L=10.0, n_orb=2),
        W.Field(kind=W.FIELD_GAUSS, amp=0.02, omega=0.0, t0=0.15, sigma=0.25, direction=(0.0, 0.6, 0.8)),
        0.04, 4, (3, 4), (0.0, 0.6, 0.8)),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    from oracle import adjoint, operators
    from paper_2210_14421_gb300 import Context
    make, field, dt, n_steps, window, d = CASES[request.param]
    wl = make()
    S = operators.System(wl)
    psi0 = S.initial_orbitals()
    psi0 /= np.linalg.norm(psi0, axis=0)
    J_ref, g_ref = adjoint.Adjoint(S).gradient(psi0, field, dt, n_steps, np.asarray(wl.occ, float),
                                               list(range(window[0], window[1] + 1)), d)
    ctx = Context(wl, krylov_tol=1e-13, k_max=40)
    return dict(wl=wl, ctx=ctx, psi0=_dev(psi0), field=field, dt=dt, n=n_steps, window=window, d=d, J=J_ref,
                g=np.asarray(g_ref))


def _run(cs, field=None, K=2, n_s=6):
    return cs["ctx"].adjoint_dipole(cs["psi0"], cs["n"], cs["dt"], field or cs["field"], cs["d"], cs["window"],
                                    checkpoint_every=K, n_quad_s=n_s)


def test_adjoint_matches_oracle(case):
    J, g = _run(case)
    assert abs(J - case["J"]) <= 1e-10 * abs(case["J"]), (J, case["J"])
    scale = np.max(np.abs(case["g"]))
    assert np.max(np.abs(g - case["g"])) <= 1e-8 * scale, (g, case["g"])


def test_adjoint_forward_is_the_magnus_step(case):
    """J of the adjoint's own forward sweep equals the window average of the
    dipoles from efe_magnus_step with the same field."""
    cs = case
    from paper_2210_14421_gb300 import Context
    ctx = Context(cs["wl"], krylov_tol=1e-13, k_max=40)
    psi = cs["psi0"].clone()
    mu = torch.zeros(3, dtype=torch.float64, device="cuda")
    acc = 0.0
    w0, w1 = cs["window"]
    for n in range(cs["n"]):
        ctx.magnus_step(psi, n * cs["dt"], cs["dt"], [cs["field"]], mu)
        if w0 <= n + 1 <= w1:
            acc += float(np.dot(cs["d"], mu.cpu().numpy())) / (w1 - w0 + 1)
    J, _ = _run(cs, n_s=1)
    assert abs(J - acc) <= 1e-11 * abs(acc), (J, acc)


def test_adjoint_matches_gpu_finite_differences(case):
    """Central differences (h = 1e-4 |theta|) of J from the CUDA forward."""
    J, g = _run(case)
    names = ["amp", "omega", "sigma"]
    for k, name in enumerate(names):
        val = getattr(case["field"], name)
        if val == 0.0:      # omega of a Gaussian pulse: J does not depend on it
            assert g[k] == 0.0
            continue
        h = 1e-4 * abs(val)
        Jp, _ = _run(case, dataclasses.replace(case["field"], **{name: val + h}), n_s=1)
        Jm, _ = _run(case, dataclasses.replace(case["field"], **{name: val - h}), n_s=1)
        fd = (Jp - Jm) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd) + 1e-13, (name, g[k], fd)


def test_checkpoint_interval_does_not_change_the_gradient(case):
    ref = _run(case, K=1)[1]
    for K in (2, 3, case["n"]):
        g = _run(case, K=K)[1]
        assert np.max(np.abs(g - ref)) <= 1e-12 * np.max(np.abs(ref)), (K, g, ref)


def test_autograd_function(case):
    from paper_2210_14421_gb300.autograd import windowed_dipole
    f = case["field"]
    theta = torch.tensor([f.amp, f.omega, f.sigma], dtype=torch.float64, requires_grad=True)
    J = windowed_dipole(theta, case["ctx"], case["psi0"], f, case["n"], case["dt"], case["d"], case["window"], 2, 6)
    (3.0 * J).backward()
    J0, g0 = _run(case)
    assert abs(J.item() - J0) <= 1e-12 * abs(J0)
    assert np.allclose(theta.grad.numpy(), 3.0 * g0, rtol=1e-12, atol=0)


def test_adjoint_rejects_bad_arguments(case):
    from paper_2210_14421_gb300 import EfeError
    cs = case
    with pytest.raises(EfeError):
        cs["ctx"].adjoint_dipole(cs["psi0"], cs["n"], cs["dt"], cs["field"], cs["d"], (1, cs["n"] + 1))
    with pytest.raises(EfeError):
        cs["ctx"].adjoint_dipole(cs["psi0"], cs["n"], cs["dt"], cs["field"], cs["d"], cs["window"], n_quad_s=0)
    with pytest.raises(EfeError):
        bad = dataclasses.replace(cs["field"], kind=W.FIELD_SINE_TRAP)
        cs["ctx"].adjoint_dipole(cs["psi0"], cs["n"], cs["dt"], bad, cs["d"], cs["window"])


def test_pair_precision_adjoint_matches_oracle(case):
    """The adjoint of a context computing in float32 pairs (pair applies, pair
    interpolation in the cross densities) reaches the oracle's gradient to the
    same 1e-8."""
    from paper_2210_14421_gb300 import EFE_PAIR, Context
    ctx = Context(case["wl"], precision=EFE_PAIR, krylov_tol=1e-13, k_max=40)
    J, g = ctx.adjoint_dipole(case["psi0"], case["n"], case["dt"], case["field"], case["d"], case["window"],
                              checkpoint_every=2, n_quad_s=6)
    assert abs(J - case["J"]) <= 1e-10 * abs(case["J"])
    assert np.max(np.abs(g - case["g"])) <= 1e-8 * np.max(np.abs(case["g"]))
