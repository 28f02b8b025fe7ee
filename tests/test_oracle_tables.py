"""Pins for the oracle's collocation and GLL tables against textbook values
and the matrices printed in Sec. 4.6 (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import tables as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_blocks(name):
    blocks, cur = [], None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line.startswith("# block"):
                cur = []
                blocks.append(cur)
            elif line and not line.startswith("#"):
                cur.append([float(v) for v in line.split()])
    return [np.array(b) for b in blocks]


def test_printed_nonequivalence_matrices():
    """Sec. 4.6: C0n_l R_l and R_l C0n_{l+1}, Radau-Right 4 -> 3 nodes."""
    c0n_r, r_c0n = _read_blocks("nonequivalence_radau_4_3.txt")
    _, _, Rt = T.time_transfers(T.radau_right(4), T.radau_right(3))
    # printed values are truncated to 5 decimals
    assert np.max(np.abs(T.c0n(3) @ Rt - c0n_r)) < 1.01e-5
    assert np.max(np.abs(Rt @ T.c0n(4) - r_c0n)) < 1.01e-5
    # and the two products differ (the proposition of Sec. 4.6)
    assert np.max(np.abs(T.c0n(3) @ Rt - Rt @ T.c0n(4))) > 0.1


def test_radau_iia_butcher():
    """cumsum of w^nn = Butcher matrix of Radau IIA (2 and 3 stages)."""
    A2 = T.w0n(T.radau_right(2))
    assert np.allclose(A2, [[5 / 12, -1 / 12], [3 / 4, 1 / 4]], atol=1e-15, rtol=0)
    s6 = math.sqrt(6.0)
    A3 = np.array([[(88 - 7 * s6) / 360, (296 - 169 * s6) / 1800, (-2 + 3 * s6) / 225],
                   [(296 + 169 * s6) / 1800, (88 + 7 * s6) / 360, (-2 - 3 * s6) / 225],
                   [(16 - s6) / 36, (16 + s6) / 36, 1 / 9]])
    assert np.allclose(T.w0n(T.radau_right(3)), A3, atol=1e-15, rtol=0)
    assert np.allclose(T.radau_right(3), [(4 - s6) / 10, (4 + s6) / 10, 1.0], atol=1e-15)


def test_lobatto_iiia_butcher():
    A3 = T.w0n(T.lobatto(3))
    assert np.allclose(A3, [[0, 0, 0], [5 / 24, 1 / 3, -1 / 24], [1 / 6, 2 / 3, 1 / 6]],
                       atol=1e-15, rtol=0)
    s5 = math.sqrt(5.0)
    assert np.allclose(T.lobatto(4), [0, (5 - s5) / 10, (5 + s5) / 10, 1], atol=1e-15)


@pytest.mark.parametrize("kind,M", [("radau_right", m) for m in range(1, 9)] +
                         [("lobatto", m) for m in range(2, 9)])
def test_wnn_row_sums_and_exactness(kind, M):
    tau = T.collocation_nodes(kind, M)
    W = T.wnn(tau)
    assert np.allclose(W.sum(axis=1), T.substeps(tau), atol=1e-14)
    # exact for polynomials of degree <= M-1: sum_i W[m,i] p(tau_i) = int p
    for deg in range(M):
        prev = np.concatenate([[0.0], tau[:-1]])
        exact = (tau ** (deg + 1) - prev ** (deg + 1)) / (deg + 1)
        assert np.allclose(W @ tau ** deg, exact, atol=1e-14)


def test_gll_textbook():
    x, w = T.gll(4)
    r = math.sqrt(3.0 / 7.0)
    assert np.allclose(x, [-1, -r, 0, r, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)
    x, w = T.gll(2)
    assert np.allclose(x, [-1, 0, 1]) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3])


@pytest.mark.parametrize("P", range(1, 11))
def test_gll_quadrature_and_derivative(P):
    x, w = T.gll(P)
    assert abs(w.sum() - 2.0) < 1e-14
    for deg in range(2 * P):          # GLL exact to degree 2P-1
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(w @ x ** deg - exact) < 1e-13
    D = T.diff_matrix(x)
    assert np.max(np.abs(D.sum(axis=1))) < 1e-12
    for deg in range(1, P + 1):
        assert np.max(np.abs(D @ x ** deg - deg * x ** (deg - 1))) < 1e-11 * P * P
    # D_00 = -P(P+1)/4, D_PP = P(P+1)/4
    assert abs(D[0, 0] + P * (P + 1) / 4) < 1e-12 and abs(D[-1, -1] - P * (P + 1) / 4) < 1e-12


@pytest.mark.parametrize("kind,Mf,Mc", [("radau_right", 5, 3), ("radau_right", 7, 5),
                                        ("lobatto", 5, 3), ("lobatto", 3, 2)])
def test_time_transfers(kind, Mf, Mc):
    tf, tc = T.collocation_nodes(kind, Mf), T.collocation_nodes(kind, Mc)
    It, Pt, Rt = T.time_transfers(tf, tc)
    assert np.allclose(Pt @ It, np.eye(Mc), atol=1e-13)
    assert np.allclose(Rt.sum(axis=0), 1.0, atol=1e-13)      # partition of unity
    for deg in range(Mc):                                   # I exact on degree < Mc
        assert np.allclose(It @ tc ** deg, tf ** deg, atol=1e-13)


@pytest.mark.parametrize("Pf,Pc", [(7, 3), (4, 2), (7, 5), (5, 3), (8, 4), (3, 3)])
def test_space_transfers(Pf, Pc):
    Ix, Px, Rx = T.space_transfers(Pf, Pc)
    xf, _ = T.gll(Pf)
    xc, _ = T.gll(Pc)
    assert np.allclose(Px @ Ix, np.eye(Pc + 1), atol=1e-13)
    for deg in range(Pc + 1):
        assert np.allclose(Ix @ xc ** deg, xf ** deg, atol=1e-13)
    assert np.allclose(Rx @ np.ones(Pf + 1), 1.0, atol=1e-13)


def test_level_cost_model_matches_printed_table():
    """The per-level costs of the paper's runtime table are DOF x M ratios of
    its discretization (the accounting of the DOF-sweep metric): 1D levels
    36 % and 11 %, 3D (h-coarsened by 2 per direction) 9 % and 0.6 %, and
    1 + N_c (0.36 + 0.11) = 1.94 fine-grid operations for N_c = 2."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "level_costs.txt")
    rows = {}
    for ln in open(path):
        if ln.strip() and not ln.startswith("#"):
            f = ln.split()
            rows[f[0]] = f[1:]
    levels = [(16, 15, 3), (32, 15, 5), (64, 15, 7)]          # (N_e, P, M), coarse to fine
    dof_m = [ne * (P + 1) * M for ne, P, M in levels]
    c2, c1 = dof_m[1] / dof_m[2], dof_m[0] / dof_m[2]
    assert round(100 * c2) == int(rows["1D_MLSDC_3_5_7"][0]) == int(rows["1D_MLSDC_5_7"][0])
    assert round(100 * c1) == int(rows["1D_MLSDC_3_5_7"][1])
    c2_3d, c1_3d = (1 / 8) * 5 / 7, (1 / 64) * 3 / 7
    assert round(100 * c2_3d) == int(rows["3D_MLSDC_3_5_7"][0]) == int(rows["3D_MLSDC_5_7"][0])
    assert math.floor(1000 * c1_3d) / 10 == float(rows["3D_MLSDC_3_5_7"][1])   # 0.67 % printed as 0.6
    Nc = 2
    printed = float(rows["three_level_1D_Nc2_fine_ops"][0])
    assert abs(1 + Nc * (0.36 + 0.11) - printed) < 1e-12
    assert abs(1 + Nc * (c2 + c1) - printed) < 0.02


@pytest.mark.parametrize("Pf,Pc", [(7, 3), (5, 3), (4, 2), (8, 4)])
def test_l2_projection(Pf, Pc):
    """The L2 solution projection is a projection (P I = identity), is the
    weighted least-squares fit under the fine GLL quadrature (checked against
    numpy's lstsq) and conserves the integral against the consistent coarse
    mass."""
    from oracle.tables import l2_projection, space_transfers
    P = l2_projection(Pf, Pc)
    Ix, _, _ = space_transfers(Pf, Pc)
    assert np.max(np.abs(P @ Ix - np.eye(Pc + 1))) < 1e-13
    xf, wf = T.gll(Pf)
    u = np.random.default_rng(Pf * 10 + Pc).standard_normal(Pf + 1)
    sw = np.sqrt(wf)
    c_ls = np.linalg.lstsq(sw[:, None] * Ix, sw * u, rcond=None)[0]
    assert np.max(np.abs(P @ u - c_ls)) < 1e-12
    ones = np.ones(Pf + 1)
    assert abs(ones @ (wf * (Ix @ (P @ u))) - wf @ u) < 1e-13


def test_cfl_delta_is_the_inflow_advection_eigenvalue():
    """The delta of the CFL definition (Sec. 8: the largest eigenvalue of the
    convection problem on the standard element with a one-sided Dirichlet
    condition, ~P^2) as the input recipe computes it, against the oracle's
    own GLL tables, and its growth like P^2."""
    import numpy as np
    from oracle.tables import diff_matrix, gll
    from paper_2504_18526_gb300 import inputs
    for P in range(1, 16):
        x, _ = gll(P)
        D = diff_matrix(x)
        want = np.max(np.abs(np.linalg.eigvals(D[1:, 1:])))
        assert abs(inputs.cfl_delta(P) - want) < 1e-9 * want
    r = [inputs.cfl_delta(P) / P ** 2 for P in (8, 12, 15)]
    assert 0.08 < min(r) and max(r) < 0.12
