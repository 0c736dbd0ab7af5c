"""Pins for the oracle's iterative method (Sec. 2.2.2): the pairwise
two-stream solutions applied through the whole column and repeated N times,
the approach that Thomas's algorithm replaces.

References, none of them the oracle's own sweep code:
  - without scattering (w0 = 0, so xi = 0) the paper notes that the upward
    and downward fluxes can be computed independently; one sweep (down, BOA,
    up) is then the exact solution, i.e. a dense LU of the block system;
  - the exact solution of the block system (dense LU) is a fixed point of
    the sweep;
  - the sweep is Gauss-Seidel on the assembled rows of Eq. 12 with each
    unknown paired with the relation that gives it, in the sweep's order;
    a dense numpy Gauss-Seidel reproduces it;
  - with scattering the sweeps converge to the block solution, monotonically.
"""
import numpy as np
import pytest

import oracle
import rt_synth
from test_oracle_pins import random_column, rel_err


def dense_matrix(A, B, Cm):
    n = A.shape[0] - 1
    M = np.zeros((2 * (n + 1), 2 * (n + 1)))
    for i in range(n + 1):
        M[2 * i:2 * i + 2, 2 * i:2 * i + 2] = B[i]
        if i > 0:
            M[2 * i:2 * i + 2, 2 * i - 2:2 * i] = A[i]
        if i < n:
            M[2 * i:2 * i + 2, 2 * i + 2:2 * i + 4] = Cm[i]
    return M


def dense_gauss_seidel(M, rhs, x, n_sweeps):
    """Gauss-Seidel on M x = rhs, unknowns x[2i] = F_up,i and x[2i+1] =
    F_dn,i (level 0 = BOA).  Row 2i+1 (second equation of block row i) gives
    F_dn,i and row 2i (first equation) gives F_up,i; the unknowns are updated
    in the order F_dn,n ... F_dn,0, F_up,0 ... F_up,n."""
    n = M.shape[0] // 2 - 1
    order = [2 * i + 1 for i in range(n, -1, -1)] + [2 * i for i in range(n + 1)]
    x = x.copy()
    for _ in range(n_sweeps):
        for k in order:
            x[k] = (rhs[k] - M[k] @ x + M[k, k] * x[k]) / M[k, k]
    return x


@pytest.mark.parametrize("iso", [False, True])
def test_one_sweep_is_exact_without_scattering(orc, iso):
    rng = np.random.default_rng(310 + iso)
    for trial in range(4):
        L = (1, 3, 7, 12)[trial]
        dtau, _, g0, Bc, Bi = random_column(rng, L, 1e-4, 20.0)
        w0 = np.zeros(L, np.float32)
        mu = rng.uniform(0.1, 1.0) if trial != 2 else -0.5
        cfg = oracle.OracleConfig(isothermal=iso, F_toa=rng.uniform(0.0, 7.0))
        A, B, Cm, D, _ = orc.assemble(cfg, dtau, w0, g0, Bc, Bi, mu, 1.2e5, 5.0)
        x = np.linalg.solve(dense_matrix(A, B, Cm), D.ravel()).reshape(-1, 2)
        up, dn, _ = orc.sweep_system(cfg, dtau, w0, g0, Bc, Bi, mu, 1.2e5, 5.0, 1)
        scale = np.abs(x).max()
        assert np.max(np.abs(up - x[:, 0])) <= 1e-12 * scale
        assert np.max(np.abs(dn - x[:, 1])) <= 1e-12 * scale
        # with scattering one sweep is not enough
        w0s = np.full(L, 0.9, np.float32)
        A, B, Cm, D, _ = orc.assemble(cfg, dtau, w0s, g0, Bc, Bi, mu, 1.2e5, 5.0)
        xs = np.linalg.solve(dense_matrix(A, B, Cm), D.ravel()).reshape(-1, 2)
        u1, d1, _ = orc.sweep_system(cfg, dtau, w0s, g0, Bc, Bi, mu, 1.2e5, 5.0, 1)
        assert max(rel_err(u1, xs[:, 0]), rel_err(d1, xs[:, 1])) > 1e-4


@pytest.mark.parametrize("iso", [False, True])
def test_block_solution_is_a_fixed_point(orc, iso):
    rng = np.random.default_rng(320 + iso)
    for L in (1, 4, 9):
        dtau, w0, g0, Bc, Bi = random_column(rng, L, 1e-3, 30.0)
        cfg = oracle.OracleConfig(isothermal=iso, F_toa=2.5)
        A, B, Cm, D, _ = orc.assemble(cfg, dtau, w0, g0, Bc, Bi, 0.4, 1e5, 5.0)
        x = np.linalg.solve(dense_matrix(A, B, Cm), D.ravel()).reshape(-1, 2)
        up, dn, _ = orc.sweep_system(cfg, dtau, w0, g0, Bc, Bi, 0.4, 1e5, 5.0, 1,
                                     up0=x[:, 0], dn0=x[:, 1])
        scale = np.abs(x).max()
        assert np.max(np.abs(up - x[:, 0])) <= 1e-12 * scale
        assert np.max(np.abs(dn - x[:, 1])) <= 1e-12 * scale


@pytest.mark.parametrize("iso", [False, True])
@pytest.mark.parametrize("n_sweeps", [1, 2, 5])
def test_sweeps_are_gauss_seidel_on_the_block_rows(orc, iso, n_sweeps):
    rng = np.random.default_rng(330 + 10 * iso + n_sweeps)
    for L in (1, 3, 6):
        dtau, w0, g0, Bc, Bi = random_column(rng, L, 1e-3, 5.0)
        mu = rng.uniform(0.1, 1.0)
        cfg = oracle.OracleConfig(isothermal=iso, F_toa=1.5)
        A, B, Cm, D, _ = orc.assemble(cfg, dtau, w0, g0, Bc, Bi, mu, 1e5, 5.0)
        n = A.shape[0] - 1
        x0 = rng.uniform(-1e4, 1e4, 2 * (n + 1))
        xg = dense_gauss_seidel(dense_matrix(A, B, Cm), D.ravel(), x0, n_sweeps).reshape(-1, 2)
        up, dn, _ = orc.sweep_system(cfg, dtau, w0, g0, Bc, Bi, mu, 1e5, 5.0, n_sweeps,
                                     up0=x0[0::2], dn0=x0[1::2])
        scale = np.abs(xg).max()
        assert np.max(np.abs(up - xg[:, 0])) <= 1e-11 * scale
        assert np.max(np.abs(dn - xg[:, 1])) <= 1e-11 * scale


@pytest.mark.parametrize("iso", [False, True])
def test_sweeps_converge_to_the_block_solution(orc, iso):
    rng = np.random.default_rng(90 + iso)
    dtau, w0, g0, Bc, Bi = random_column(rng, 6, 1e-3, 3.0, w_hi=0.9)
    cfg = oracle.OracleConfig(isothermal=iso)
    A, B, Cm, D, _ = orc.assemble(cfg, dtau, w0, g0, Bc, Bi, 0.5, 1e5, 5.0)
    x = np.linalg.solve(dense_matrix(A, B, Cm), D.ravel()).reshape(-1, 2)
    errs = []
    for N in (1, 10, 50, 200, 2000):
        up, dn, _ = orc.sweep_system(cfg, dtau, w0, g0, Bc, Bi, 0.5, 1e5, 5.0, N)
        errs.append(max(rel_err(up, x[:, 0]), rel_err(dn, x[:, 1])))
    assert all(a >= b for a, b in zip(errs[:-1], errs[1:]))
    assert errs[0] > 1e-3 and errs[-1] < 1e-10


def test_batch_sweeps_reduce_to_thomas(orc):
    """Whole batches: one sweep equals the block solve when nothing scatters;
    many sweeps equal it with scattering (spectral sums, net flux and
    heating included)."""
    cols = rt_synth.generate([5, 3], [4, 6], 2, seed=7, optics="uniform")
    base = oracle.OracleConfig(wn_min=cols.consts["wn_min"], wn_max=cols.consts["wn_max"])
    ref = orc.solve_columns(base, cols)
    from dataclasses import replace
    many = orc.solve_columns(replace(base, n_sweeps=4000), cols)
    for k in ("F_up", "F_down", "F_net", "Q", "F_up_toa"):
        scale = np.abs(ref[k]).max()
        assert np.max(np.abs(many[k] - ref[k])) <= 1e-9 * scale, k
    few = orc.solve_columns(replace(base, n_sweeps=2), cols)
    assert np.max(np.abs(few["F_up"] - ref["F_up"])) > 1e-6 * np.abs(ref["F_up"]).max()
    cols0 = replace(cols, w0=np.zeros_like(cols.w0))
    ref0 = orc.solve_columns(base, cols0)
    one = orc.solve_columns(replace(base, n_sweeps=1), cols0)
    for k in ("F_up", "F_down", "F_net", "Q"):
        scale = np.abs(ref0[k]).max()
        assert np.max(np.abs(one[k] - ref0[k])) <= 1e-11 * scale, k
    # the branch counters do not depend on the solver
    assert many["stats"] == ref["stats"]
