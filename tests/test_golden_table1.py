"""Golden fixture: Table 1's 17 recycling strategies (tests/golden/table1_strategies.tsv).

Each row's side, vector type and size is mapped from its words (not from the acronym), then
checked against (1) the strategy grammar of the library and (2) what the checker's refresh
selects, the latter against spectra computed here independently: eigenvalues of W~^T H W~ for
Ritz vectors, of the pencil ((H W~)^T H W~, (H W~)^T W~) for harmonic Ritz vectors, singular
values of (J W~)(W~^T H W~)^{-1} for Ritz generalized singular vectors, and for the two
full-space rows (Eig-S, GSVD-L(R): W = I) the spectrum of H and of J H^{-1}."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import recycle as rc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_strategies.tsv")
KIND = {"eigenvectors": "eig", "generalized singular vectors": "gsvd", "Ritz vectors": "ritz",
        "harmonic Ritz vectors": "hritz", "Ritz generalized singular vectors": "rgsv"}
SIZE = {"small": "S", "large": "L", "small & large": "M"}
SIDE = {"-": None, "right": "R", "left": "L", "left & right": "M"}


def rows():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            acr, side, vec, size = line.rstrip("\n").split("\t")
            out.append((acr, SIDE[side], KIND[vec], SIZE[size]))
    return out


ROWS = rows()


def expected(values_ascending, s, size):
    v = np.asarray(values_ascending)
    if size == "S":
        return v[:s]
    if size == "L":
        return v[-s:]
    return np.concatenate([v[:s // 2], v[-(s // 2):]])     # half of each (s even here)


def problem(seed=0, n=14, t=8, p=11):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    H = (Q * np.linspace(0.5, 40.0, n)) @ Q.T
    J = rng.standard_normal((p, n))
    Wt, _ = np.linalg.qr(rng.standard_normal((n, t)))
    return H, J, Wt


def test_table_has_the_17_rows():
    assert len(ROWS) == 17
    assert len({r[0] for r in ROWS}) == 17


@pytest.mark.parametrize("acr,side,kind,size", ROWS, ids=[r[0] for r in ROWS])
def test_grammar_matches_table(acr, side, kind, size):
    from paper_2412_08264_gb300.strategy import parse
    if kind in ("eig", "gsvd"):
        with pytest.raises(ValueError):     # full-space strategies need the dense Hessian
            parse(acr)
        return
    st = parse(acr)
    assert (st.kind, st.size) == (kind, size)
    if kind == "rgsv":
        assert st.side == side
    else:
        assert side is None
    assert st.acronym() == acr


@pytest.mark.parametrize("acr,side,kind,size", ROWS, ids=[r[0] for r in ROWS])
def test_checker_selects_what_the_table_says(acr, side, kind, size):
    H, J, Wt = problem()
    s = 4
    if kind == "eig":                                   # W = I: eigenvectors of H itself
        I = np.eye(H.shape[0])
        Qs, lam = rc.ritz(I, H, s, size)
        np.testing.assert_allclose(lam, expected(np.linalg.eigvalsh(H), s, size), rtol=1e-12)
        np.testing.assert_allclose(H @ Qs, Qs * lam, atol=1e-10)
        return
    if kind == "gsvd":                                  # W = I: GSVD of (J, H)
        I = np.eye(H.shape[0])
        Y, Z, mu = rc.rgsv(I, H, J, s, size, side)
        sv = np.sort(np.linalg.svd(J @ np.linalg.inv(H), compute_uv=False))
        sv = np.concatenate([np.zeros(H.shape[0] - len(sv)), sv]) if len(sv) < H.shape[0] else sv
        np.testing.assert_allclose(mu, expected(sv, s, size), rtol=1e-10)
        return
    HW = H @ Wt
    T = Wt.T @ HW
    if kind == "ritz":
        Q, lam = rc.ritz(Wt, HW, s, size)
        np.testing.assert_allclose(lam, expected(np.linalg.eigvalsh(0.5 * (T + T.T)), s, size), rtol=1e-12)
        np.testing.assert_allclose(T @ Q, Q * lam, atol=1e-10)          # Ritz pairs of W~^T H W~
    elif kind == "hritz":
        R, th = rc.harmonic_ritz(Wt, HW, s, size)
        pencil = np.sort(sla.eigvals(HW.T @ HW, HW.T @ Wt).real)
        np.testing.assert_allclose(th, expected(pencil, s, size), rtol=1e-10)
        np.testing.assert_allclose(HW.T @ HW @ R, (HW.T @ Wt) @ R * th, atol=1e-8 * np.abs(th).max())
    else:
        Y, Z, mu = rc.rgsv(Wt, HW, J @ Wt, s, size, side)
        sv = np.sort(np.linalg.svd(J @ Wt @ np.linalg.inv(T), compute_uv=False))
        np.testing.assert_allclose(mu, expected(sv, s, size), rtol=1e-10)
        Ts = 0.5 * (T + T.T)
        if side == "L":                                 # W~ V_H: orthonormal coefficient columns
            np.testing.assert_allclose(Y.T @ Y, np.eye(s), atol=1e-10)
        elif side == "R":                               # W~ X: T X = V_H D_H has orthogonal columns
            G = (Ts @ Y).T @ (Ts @ Y)
            np.testing.assert_allclose(G - np.diag(np.diag(G)), 0.0, atol=1e-10)
            assert np.linalg.norm(Y.T @ Y - np.eye(s)) > 1e-3           # and is not itself orthonormal
        else:                                           # both sides: the average of the two
            YL, _, _ = rc.rgsv(Wt, HW, J @ Wt, s, size, "L")
            YR, _, _ = rc.rgsv(Wt, HW, J @ Wt, s, size, "R")
            np.testing.assert_allclose(Y, 0.5 * (YL + YR), atol=1e-12)
