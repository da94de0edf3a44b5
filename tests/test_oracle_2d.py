"""Pins of the 2D oracle (oracle/pn2d.py, section "2D checkerboard"): the 2D
system must equal the 3D oracle's system with a z-periodic wrap and
z-independent data, restricted to the l + m even moments, both as an
operator and in its solution, and the l + m odd moments of that 3D solution
must vanish."""
import numpy as np
import pytest

import pn_inputs
from oracle import pn, pn2d
from oracle.sh import lm_list


def _bcast(a2, R):
    a2 = np.asarray(a2, dtype=np.float64)
    return np.broadcast_to(a2, (R,) + a2.shape).copy()


def _data(N, R, seed):
    rng = np.random.default_rng(seed)
    st2 = rng.uniform(0.5, 4.0, (R, R))
    al2 = rng.uniform(0.3, 0.95, (R, R))
    q2 = rng.uniform(0.0, 1.0, (R, R))
    return st2, al2, q2, 0.3


@pytest.mark.parametrize("N,R", [(1, 5), (3, 5), (5, 4)])
def test_2d_operator_equals_z_periodic_3d_operator(N, R):
    st2, al2, q2, g = _data(N, R, N)
    lay2, A2, b2 = pn2d.assemble_2d(N, R, st2, al2, g, q2)
    S3 = pn.assemble(N, R, pn.Medium(_bcast(st2, R), _bcast(al2, R), g, _bcast(q2, R)), periodic=(False, False, True))
    rng = np.random.default_rng(100 + N)
    u2 = [rng.standard_normal(s) for s in lay2.shapes]
    parts3 = []
    for k3, (l, m) in enumerate(lm_list(N)):
        if (l + m) % 2:
            parts3.append(np.zeros(S3.layout.shapes[k3]))
        else:
            parts3.append(_bcast(u2[lay2.k3.index(k3)], R))
    y3 = S3.layout.split(S3.A @ S3.layout.join(parts3))
    y2 = lay2.split(A2 @ lay2.join(u2))
    scale = max(np.abs(y).max() for y in y2)
    for k3, (l, m) in enumerate(lm_list(N)):
        if (l + m) % 2:
            assert np.abs(y3[k3]).max() <= 1e-13 * scale
        else:
            for iz in range(R):
                np.testing.assert_allclose(y3[k3][iz], y2[lay2.k3.index(k3)], rtol=0, atol=1e-13 * scale)
    # right-hand side: Q00 on the centre grid only
    b3 = S3.layout.split(S3.b)
    np.testing.assert_allclose(b3[0][0], lay2.split(b2)[0], rtol=0, atol=0)


@pytest.mark.parametrize("N,R", [(1, 6), (3, 5)])
def test_2d_solution_equals_z_periodic_3d_solution(N, R):
    st2, al2, q2, g = _data(N, R, 10 + N)
    lay2, A2, b2 = pn2d.assemble_2d(N, R, st2, al2, g, q2)
    u2 = lay2.split(pn2d.solve_direct_2d(A2, b2))
    S3 = pn.assemble(N, R, pn.Medium(_bcast(st2, R), _bcast(al2, R), g, _bcast(q2, R)), periodic=(False, False, True))
    u3 = S3.layout.split(pn.solve_direct(S3))
    scale = np.abs(u2[0]).max()
    assert scale > 1e-3
    for k3, (l, m) in enumerate(lm_list(N)):
        if (l + m) % 2:
            assert np.abs(u3[k3]).max() <= 1e-12 * scale
        else:
            for iz in range(R):
                np.testing.assert_allclose(u3[k3][iz], u2[lay2.k3.index(k3)], rtol=0, atol=1e-11 * scale)


def test_2d_moment_source_equals_3d():
    """A source given as moments (all l + m even moments nonzero)."""
    N, R = 3, 4
    st2, al2, _, g = _data(N, R, 21)
    lay2 = pn2d.Layout2D(N, R)
    rng = np.random.default_rng(22)
    Q2 = rng.uniform(-1.0, 1.0, (lay2.K, R, R))
    _, A2, b2 = pn2d.assemble_2d(N, R, st2, al2, g, Q2)
    Q3 = np.zeros(((N + 1) ** 2, R, R, R))
    for k2, k3 in enumerate(lay2.k3):
        Q3[k3] = _bcast(Q2[k2], R)
    S3 = pn.assemble(N, R, pn.Medium(_bcast(st2, R), _bcast(al2, R), g, Q3), periodic=(False, False, True))
    b3 = S3.layout.split(S3.b)
    for k2, k3 in enumerate(lay2.k3):
        np.testing.assert_allclose(b3[k3][0], lay2.split(b2)[k2], rtol=1e-15, atol=1e-15)


def test_planted_sign_error_in_y_couplings_is_caught(monkeypatch):
    """Flipping the sign of A_y inside the 2D assembler breaks the operator
    equality with the 3D oracle."""
    orig = pn2d.coupling_matrices

    def flipped(N):
        A = orig(N).copy()
        A[1] *= -1.0
        return A
    monkeypatch.setattr(pn2d, "coupling_matrices", flipped)
    with pytest.raises(AssertionError):
        test_2d_operator_equals_z_periodic_3d_operator(3, 4)


def test_2d_layout_counts():
    for N in range(8):
        lay = pn2d.Layout2D(N, 4)
        assert lay.K == (N + 1) * (N + 2) // 2
        assert all((l + m) % 2 == 0 for l, m in lay.lm)


def test_checkerboard_input():
    st, al, Q = pn_inputs.checkerboard_2d(71)
    assert st.shape == (71, 71)
    # 7 x 7 unit blocks; 24 absorbing (i + j odd), 25 scattering; source in block (3, 3)
    c = np.floor((np.arange(71) + 0.5) * 7 / 71).astype(int)
    assert c[0] == 0 and c[-1] == 6 and np.all(np.diff(c) >= 0)
    absorbing = al == 0.0
    assert np.all(st[absorbing] == 70.0) and np.all(st[~absorbing] == 7.0)
    blocks = {(c[i], c[j]) for i in range(71) for j in range(71) if absorbing[i, j]}
    assert len(blocks) == 24 and (3, 3) not in blocks
    src = Q > 0
    assert {(c[i], c[j]) for i in range(71) for j in range(71) if src[i, j]} == {(3, 3)}
    assert np.all(al[src] == 1.0)
