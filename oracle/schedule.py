"""Algorithm 3 (finite-size parameter schedule), exact rational arithmetic.

Test infrastructure only (part of the oracle).  Follows Methods, "Finite-size
parameter schedule" (Algorithm 3) and SI "Analysis of the finite-size parameter
schedule":

    phibar_k      = phi_min + (1 - phi_min) q^(k-1)
    Phi_{k+1}(b)  = phi_k - (phi_k + 2) d_k / ((phi_k + 1) d_k + phi_k b)
    d_1 = w_max + 1, phi_1 = 1
    b_k = smallest integer with b >= d_k, phi_k > 2 d_k / b, Phi_{k+1}(b) >= phibar_{k+1}
    phi_{k+1} = Phi_{k+1}(b_k),  d_{k+1} = 3 d_k + 4 b_k + 2 w_max

All distances are in the decoder's internal units (twice the integer edge
weights), so w_max here is the largest internal weight.
"""

from __future__ import annotations

import math
from fractions import Fraction


def phibar(k: int, q: Fraction, phi_min: Fraction) -> Fraction:
    return phi_min + (1 - phi_min) * q ** (k - 1)


def big_phi(phi_k: Fraction, d_k: int, b) -> Fraction:
    return phi_k - (phi_k + 2) * d_k / ((phi_k + 1) * d_k + phi_k * b)


def admissible(phi_k: Fraction, d_k: int, b: int, target: Fraction) -> bool:
    return b >= d_k and b > 0 and phi_k > Fraction(2 * d_k, b) and big_phi(phi_k, d_k, b) >= target


def alg3(w_max: int, q=Fraction(1, 10), phi_min=Fraction(1, 100), levels: int = 6, d1=None, b1=None):
    """Return (d, b, phi) lists for levels 1..levels (index 0 is level 1).

    d1 / b1 replace level 1's diameter / buffer (b1 must be admissible for
    level 1, it need not be the smallest); later levels follow by the same
    recursion."""
    q = Fraction(q)
    phi_min = Fraction(phi_min)
    d = [w_max + 1 if not d1 else int(d1)]
    phi = [Fraction(1)]
    b = []
    for k in range(1, levels + 1):
        dk, pk = d[-1], phi[-1]
        target = phibar(k + 1, q, phi_min)
        if not pk > target:
            raise ValueError("schedule has no admissible b at level %d" % k)
        if k == 1 and b1:
            bk = int(b1)
            if not admissible(pk, dk, bk, target):
                raise ValueError("b1 = %d is not admissible for d1 = %d" % (bk, dk))
            b.append(bk)
            phi.append(big_phi(pk, dk, bk))
            d.append(3 * dk + 4 * bk + 2 * w_max)
            continue
        # b > 2 d_k / phi_k
        lo1 = math.floor(Fraction(2 * dk) / pk) + 1
        # Phi(b) >= target  <=>  b >= ((phi+2) d / (phi - target) - (phi+1) d) / phi
        x = (((pk + 2) * dk) / (pk - target) - (pk + 1) * dk) / pk
        lo2 = math.ceil(x)
        bk = max(dk, lo1, lo2, 1)
        assert admissible(pk, dk, bk, target)
        assert bk - 1 < 1 or not admissible(pk, dk, bk - 1, target)
        b.append(bk)
        phi.append(big_phi(pk, dk, bk))
        d.append(3 * dk + 4 * bk + 2 * w_max)
    return d[:levels], b, phi[:levels]
