"""Oracle blob-level random finite difference (Sec. 3, eq. RFDcenter with
B = M and Delta P = Delta Q = W).  TEST INFRASTRUCTURE.

drift = (1/delta) [M(r + delta/2 W) - M(r - delta/2 W)] W;
its mean over W ~ N(0, I) is div M + O(delta^2) (eq. RFDB with kT = 1).
"""
from . import mobility


def rfd_drift(r, W, delta, prm: mobility.Params):
    rp = r + 0.5 * delta * W
    rm = r - 0.5 * delta * W
    return (mobility.apply(rp, W, prm) - mobility.apply(rm, W, prm)) / delta
