"""D2Q37 velocity set and quadrature weights for the oracle.

TEST INFRASTRUCTURE ONLY: part of the CPU oracle. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may use it.

The paper names a 37-velocity two-dimensional lattice whose populations hop at
most three sites per step (Sec. "Lattice Boltzmann methods", Eq. discrete and
Fig. streamscheme) but prints neither the velocity vectors nor the weights.
Reading used here:

* velocities: every integer vector c with |c|^2 <= 10.  That is exactly 37
  vectors in 8 shells (|c|^2 in {0,1,2,4,5,8,9,10}) with |c_x|,|c_y| <= 3;
  26 of them cross a vertical boundary, which is the count the paper gives
  for the populations exchanged per boundary site (Sec. "1-D Splitting").
* thermal velocities xi_l = s * c_l with one common scale s.
* weights: one weight per shell.  The 8 weights and s solve the 9 moment
  conditions sum_l w_l xi_x^i xi_y^j = E[X^i] E[Y^j] (X, Y independent
  standard normal) for (i, j) in {(0,0),(2,0),(4,0),(2,2),(6,0),(4,2),(8,0),
  (6,2),(4,4)}.  With the square symmetry of the set this makes the
  quadrature exact for every monomial of degree <= 9, which the 4th-order
  Hermite equilibrium needs (Eq. MASTERSHIFT3 expanded to 4th order).

The solve is Newton's method on all 9 unknowns in 50-digit ``decimal``
arithmetic (standard library only), so the weights are correct to far below
one FP64 ulp before they are rounded.
"""
from decimal import Decimal, getcontext

SHELL_C2 = (0, 1, 2, 4, 5, 8, 9, 10)
MOMENT_ORDERS = ((0, 0), (2, 0), (4, 0), (2, 2), (6, 0), (4, 2), (8, 0), (6, 2), (4, 4))


def velocity_set():
    """The 37 integer hops c_l = (cx, cy) with |c|^2 <= 10, in enumeration order."""
    return [(cx, cy) for cx in range(-3, 4) for cy in range(-3, 4) if cx * cx + cy * cy <= 10]


def gaussian_moment(k):
    """E[Z^k] for a standard normal Z: 0 for odd k, (k-1)!! for even k."""
    if k % 2:
        return 0
    m = 1
    for i in range(k - 1, 0, -2):
        m *= i
    return m


def _solve(a, b):
    """Gaussian elimination with partial pivoting on Decimal lists."""
    n = len(b)
    m = [row[:] + [b[i]] for i, row in enumerate(a)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(m[r][col]))
        m[col], m[piv] = m[piv], m[col]
        for r in range(col + 1, n):
            f = m[r][col] / m[col][col]
            for c in range(col, n + 1):
                m[r][c] -= f * m[col][c]
    x = [Decimal(0)] * n
    for r in range(n - 1, -1, -1):
        acc = m[r][n]
        for c in range(r + 1, n):
            acc -= m[r][c] * x[c]
        x[r] = acc / m[r][r]
    return x


def solve_weights(digits=50, s_start="1.2"):
    """Return (s, [w_shell0..w_shell7]) as Decimals.

    Unknowns x = (w_0..w_7, s).  Residuals
    F_e = s^(i+j) * sum_k w_k B[e][k] - E[X^i] E[Y^j], with the integer shell
    sums B[e][k] = sum_{l in shell k} cx^i cy^j.
    """
    getcontext().prec = digits
    vel = velocity_set()
    B = [[sum(cx ** i * cy ** j for cx, cy in vel if cx * cx + cy * cy == c2) for c2 in SHELL_C2]
         for i, j in MOMENT_ORDERS]
    rhs = [Decimal(gaussian_moment(i) * gaussian_moment(j)) for i, j in MOMENT_ORDERS]
    s = Decimal(s_start)
    # start: weights from the 8 conditions other than (8, 0) at the starting
    # scale (the 8 conditions without (4, 4) are linearly dependent in w)
    start = [e for e, ij in enumerate(MOMENT_ORDERS) if ij != (8, 0)]
    w = _solve([[s ** sum(MOMENT_ORDERS[e]) * B[e][k] for k in range(8)] for e in start],
               [rhs[e] for e in start])
    tol = Decimal(10) ** (-(digits - 8))
    for _ in range(100):
        F, J = [], []
        for e, (i, j) in enumerate(MOMENT_ORDERS):
            n = i + j
            lin = sum(w[k] * B[e][k] for k in range(8))
            F.append(s ** n * lin - rhs[e])
            row = [s ** n * B[e][k] for k in range(8)]
            row.append(n * s ** (n - 1) * lin if n > 0 else Decimal(0))
            J.append(row)
        d = _solve(J, F)
        w = [w[k] - d[k] for k in range(8)]
        s = s - d[8]
        if max(abs(v) for v in d) < tol:
            break
    else:
        raise RuntimeError("quadrature Newton iteration did not converge")
    return s, w


_CACHE = {}


def weights_fp64():
    """(s, w_shell[8]) rounded to the nearest FP64 values."""
    if "fp64" not in _CACHE:
        s, w = solve_weights()
        _CACHE["fp64"] = (float(s), [float(x) for x in w])
    return _CACHE["fp64"]
