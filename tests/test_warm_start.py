"""The premise of where the global solves start (a reading of Eq. 8's solve,
which the paper leaves to a library solver): along the loop's trajectory,
x_i + (x_i - x_(i-1)) is a closer guess for x_(i+1) than x_i.  Checked on the
oracle's own systems, independently of the CUDA path: after the first few
iterations from rest the first residual of each global step, relative to its
right-hand side, is several times smaller from the extrapolated start.  The
solution itself does not depend on the start (the solves stop at the same
relative residual); only the number of CG iterations does."""
import numpy as np

from oracle import global_step, loop
from paper_2203_02054_gb300 import synth


def _systems(m, n_iters, monkeypatch):
    """The free-row systems A x = rhs of the oracle's global steps, with the
    positions x_i each one starts from."""
    out = []
    solve = global_step.solve

    def recording_solve(A, b, X, fixed):
        free = ~fixed.astype(bool)
        Aff = A[free][:, free].tocsr()
        rhs = b[free] - A[free][:, ~free] @ X[~free]
        out.append((Aff, rhs, X[free].copy()))
        return solve(A, b, X, fixed)

    monkeypatch.setattr(loop.global_step, "solve", recording_solve)
    loop.run_mesh(m, n_iters=n_iters)
    return out


def test_extrapolated_start_lowers_the_first_residual(monkeypatch):
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4, seed=7, n_iters=20)
    sys_ = _systems(m, 20, monkeypatch)
    assert len(sys_) == 20
    ratios = []
    for i in range(1, len(sys_)):
        A, rhs, x = sys_[i]
        step = x - sys_[i - 1][2]
        r_plain = np.linalg.norm(rhs - A @ x)
        r_extra = np.linalg.norm(rhs - A @ (x + step))
        ratios.append(r_plain / r_extra)
    late = np.array(ratios[4:])          # iterations 5..19
    assert np.all(late > 1.0), ratios
    assert np.median(late) >= 3.0, ratios
    # from rest the direction still turns quickly: early on the plain start is
    # the better one, which the solves absorb with a few more CG iterations
    assert ratios[0] < 1.0, ratios
