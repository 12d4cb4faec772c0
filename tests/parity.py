"""Element-by-element comparison of GPU results with the CPU oracle.

Tolerance: every eigenvalue and every eigenvector component within relative
error 10 n eps64 (eps64 = 2^-53) of the oracle.  Two refinements, both from
the oracle's own error bounds rather than from the GPU:
  * an eigenvalue whose oracle absolute error bound exceeds that (an exact zero
    eigenvalue, where relative error is undefined) is compared absolutely;
  * components below DBL_MIN are compared absolutely at DBL_MIN * tol.
"""
import numpy as np

EPS64 = 2.0 ** -53
DBL_MIN = np.finfo(np.float64).tiny


def tolerance(n, factor=10.0):
    return factor * n * EPS64


def widened(orc, n, factor=10.0):
    """Mask of the eigenvalues whose comparison the oracle's own bound widens:
    where 4 abserr exceeds factor n eps64 |lambda|, lam_errors divides by the
    bound instead of |lambda|.  Full-size checks assert that this mask is
    empty, so that no comparison there relaxes silently; the only expected
    member elsewhere is an exactly zero eigenvalue (relative error undefined)."""
    lam_or = np.abs(orc["lam"])
    absb = orc.get("abserr", np.zeros_like(lam_or))
    return 4 * absb / tolerance(n, factor) > lam_or


def lam_errors(lam_gpu, orc, n):
    lam_or = orc["lam"]
    scale = np.abs(lam_or)
    absb = orc.get("abserr", np.zeros_like(lam_or))
    err = np.abs(lam_gpu - lam_or)
    # error in units of n*eps64, relative where meaningful
    denom = np.maximum(scale, 4 * absb / tolerance(n))
    denom = np.where(denom == 0, 1.0, denom)
    return err / denom / (n * EPS64)


def vec_errors(V_gpu, V_or, n):
    a = np.abs(V_or)
    err = np.abs(V_gpu - V_or)
    denom = np.maximum(a, DBL_MIN)
    return err / denom / (n * EPS64)


def assert_parity(lam_gpu, V_gpu, orc, n, factor=10.0, cols=None, what=""):
    """Raise with a readable summary if any eigenvalue/component is out of tolerance."""
    le = lam_errors(lam_gpu, orc, n)
    worst_l = float(np.max(le)) if le.size else 0.0
    msgs = []
    if worst_l > factor:
        k = int(np.argmax(le))
        msgs.append(f"eigenvalue {k}: gpu {lam_gpu[k]!r} oracle {orc['lam'][k]!r} "
                    f"err {worst_l:.3g} n*eps")
    worst_v = 0.0
    if V_gpu is not None:
        ve = vec_errors(V_gpu, orc["V"], n)
        worst_v = float(np.max(ve)) if ve.size else 0.0
        if worst_v > factor:
            r, k = np.unravel_index(int(np.argmax(ve)), ve.shape)
            kk = k if cols is None else cols[k]
            msgs.append(f"vector comp ({r},{kk}): gpu {V_gpu[r, k]!r} oracle "
                        f"{orc['V'][r, k]!r} err {worst_v:.3g} n*eps")
    assert not msgs, f"{what} parity failed (tol {factor} n eps64): " + "; ".join(msgs)
    return worst_l, worst_v
