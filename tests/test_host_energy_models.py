"""Host models of two exact-integer steps of the GPU path, restated in Python integers and checked
against the oracle and numpy. They pin the arguments the CUDA code relies on; the kernels
themselves are compared with the oracle in the GPU tests.

* Initial energy from the fields (Eq. 1): with f = J s + h, sum_i s_i f_i counts every pair term
  twice and every field term once, so E = (sum_i s_i f_i + sum_i s_i h_i) / 2. In the fixed-point
  form the fused search kernel uses, aq_i = -2 s_i fq_i, so s_i fq_i = -aq_i / 2; both halvings
  are exact (aq_i is even, the sum is twice an integer).
* Fixed-point couplings: Jq = J 2^q rounded to the nearest integer, ties to even, formed from the
  FP64 bit pattern with integer operations only (significand, exponent, a right shift with a
  round-half-even correction), equal to numpy's rint(ldexp(J, q)).
"""
import struct

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import inputs as I


def fixed_point_rn(x: float, q: int) -> int:
    """x 2^q rounded to nearest, ties to even, from the bit pattern of x (integers only)."""
    u = struct.unpack("<Q", struct.pack("<d", x))[0]
    e = (u >> 52) & 0x7FF
    m = u & ((1 << 52) - 1)
    if e == 0 and m == 0:
        return 0
    if e != 0:
        m |= 1 << 52
    sh = (1 if e == 0 else e) - 1075 + q
    if sh >= 0:
        v = m << sh
    elif sh <= -54:
        v = 0
    else:
        r = -sh
        t, rem, half = m >> r, m & ((1 << r) - 1), 1 << (r - 1)
        v = t + (1 if rem > half or (rem == half and t & 1) else 0)
    return -v if u >> 63 else v


@pytest.mark.parametrize("ens,n,seed", [("gaussian", 40, 1), ("gaussian", 131, 2), ("pm1", 64, 3), ("uniform", 77, 4)])
def test_initial_energy_from_exact_fields(ens, n, seed):
    J, h = I.instance(ens, n, seed=seed)
    q = 0 if ens == "pm1" else I.GRID_BITS
    Jq = [[fixed_point_rn(float(J[i, j]), q) for j in range(n)] for i in range(n)]
    hq = [fixed_point_rn(float(h[i]), q) for i in range(n)]
    phi = I.random_states(n, 6, seed=seed + 100)
    sig = I.unpack_bits(phi, n)                  # sigma_i = 1 <=> s_i = -1
    E_ref = O.energies(J, h, phi)
    for r in range(phi.shape[0]):
        s = [-1 if sig[r, i] else 1 for i in range(n)]
        fq = [sum(Jq[i][j] * s[j] for j in range(n)) + hq[i] for i in range(n)]
        aq = [-2 * s[i] * fq[i] for i in range(n)]
        assert all(a % 2 == 0 for a in aq)
        tot = sum(-a // 2 for a in aq) + sum(s[i] * hq[i] for i in range(n))
        assert tot % 2 == 0
        Eq = tot // 2
        # the direct double sum over the pairs and the fields, in integers
        direct = sum(Jq[i][j] * s[i] * s[j] for i in range(n) for j in range(i + 1, n)) + sum(hq[i] * s[i] for i in range(n))
        assert Eq == direct
        assert np.ldexp(float(Eq), -q) == E_ref[r]   # grid inputs: the oracle's FP64 energy is exact


def test_fixed_point_conversion_matches_rint_ldexp():
    rng = np.random.default_rng(7)
    xs = list(rng.standard_normal(3000))
    xs += [float(np.ldexp(np.round(v * 1e6), -32)) for v in rng.standard_normal(1000)]                 # grid values
    xs += [float(np.ldexp(k + 0.5, -q)) * sg for k, q, sg in zip(rng.integers(0, 4096, 1000), rng.integers(0, 50, 1000),
                                                                  rng.choice([-1.0, 1.0], 1000))]      # exact ties
    xs += [float(np.ldexp(v, -int(e))) for v, e in zip(rng.standard_normal(1000), rng.integers(900, 1080, 1000))]  # tiny, subnormal
    xs += [0.0, -0.0, 5e-324, -5e-324, 1.0, -15.0, 2.5, 3.5, -2.5]
    for q in (0, 1, 17, 32, 51):
        for x in xs:
            y = np.ldexp(x, q)
            if abs(y) >= 2.0 ** 62:
                continue
            assert fixed_point_rn(x, q) == int(np.rint(y)), (x, q)
