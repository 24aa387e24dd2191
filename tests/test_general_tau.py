"""Why the scheme keeps tau = dt (Sec. 3, eq. f-eq fixes tau = dt).

For a relaxation rate omega = dt / tau other than 1 the collision keeps a
fraction (1 - omega) of the non-equilibrium part, so the five distributions
carry state of their own.  A Fourier mode exp(i k.x) of the state (f^0..f^4,
w) is multiplied each step by a 6 x 6 amplification matrix:
    f0' = (1 - omega) f0 + omega (sum_a f^a - 4 G w)
    fk' = exp(-i k.c_k) ((1 - omega) fk + omega G w)       (pull from x - c_k)
    w'  = w + dt sum_a f^a'
With omega = 1 every eigenvalue has modulus 1 for G <= 1/2 (the leapfrog
bound g dt <= 1/2 that lbm_create enforces) and the scheme is neutral; with
any omega != 1 and any scale G > 0 of the equilibrium some mode has modulus
above 1, so the general-tau distribution form grows without bound.  The
oracle, which steps the distribution form literally, shows the same growth.
This is the reason the CUDA library accepts only omega = 1."""
import numpy as np
import pytest

from paper_2206_12412_gb300 import workloads as W


def _spectral_radius(omega, G, nk=25):
    worst = 0.0
    for kx in np.linspace(0.0, np.pi, nk):
        for ky in np.linspace(0.0, np.pi, nk):
            if kx == 0.0 and ky == 0.0:
                continue        # the uniform mode: a Jordan block of eigenvalue 1 (rigid drift)
            ph = [1.0, np.exp(-1j * kx), np.exp(-1j * ky), np.exp(1j * kx), np.exp(1j * ky)]
            M = np.zeros((6, 6), complex)
            M[0, :5] = omega
            M[0, 0] += 1.0 - omega
            M[0, 5] = -4.0 * omega * G
            for a in range(1, 5):
                M[a, a] = ph[a] * (1.0 - omega)
                M[a, 5] = ph[a] * omega * G
            M[5, :] = M[:5, :].sum(axis=0)
            M[5, 5] += 1.0
            worst = max(worst, float(np.abs(np.linalg.eigvals(M)).max()))
    return worst


@pytest.mark.parametrize("g", [0.05, 0.25, 0.5])
def test_unit_omega_is_neutral_up_to_the_leapfrog_bound(g):
    assert _spectral_radius(1.0, g) <= 1.0 + 1e-7


def test_unit_omega_beyond_the_leapfrog_bound_grows():
    assert _spectral_radius(1.0, 0.55) > 1.05


@pytest.mark.parametrize("omega", [0.5, 0.9, 0.99, 1.01, 1.1, 1.5])
@pytest.mark.parametrize("G", [0.01, 0.1, 0.25])
def test_every_other_omega_grows(omega, G):
    assert _spectral_radius(omega, G) > 1.0 + 1e-5


def test_oracle_distribution_form_grows_for_omega_not_one(oracle_mod):
    nx = ny = 32
    out = {}
    for omega in (1.0, 0.9):
        p = W.base_problem(nx, ny, edges=("periodic", "periodic", "periodic", "periodic"))
        p["omega"] = omega
        o = oracle_mod.Oracle(p)
        w0, wd0 = W.random_state(nx, ny, seed=3)
        o.set_fields(w0, wd0 * 0.0)
        o.step(3000)
        w, _ = o.fields()
        out[omega] = np.abs(w - w.mean()).max() / np.abs(w0 - w0.mean()).max()
        o.close()
    assert out[1.0] < 3.0
    assert out[0.9] > 1e3
