"""Exact one-axis-twisting dynamics in the symmetric (Dicke) subspace (Sec. II.B, Eqs. 12-15).

TEST INFRASTRUCTURE ONLY: imported by tests and the benchmark's OAT mode as the exact
reference; never by the product path.

H = chi (S^z)^2 with S^a = sum_i S^a_i (Eq. 12) conserves the total spin, and the initial
state, every spin along +x, lies in the S = N/2 multiplet.  In the Dicke basis |S, m>,
m = -S..S, the initial amplitudes are 2^(-N/2) sqrt(binom(N, S + m)) (the +x product state
expanded over the configurations with S + m up spins), and the evolution multiplies them by
exp(-i chi t m^2).  The total-spin moments follow from the (N + 1)-dimensional spin matrices:
  S^z |m> = m |m>,  S^+ |m> = sqrt(S(S + 1) - m(m + 1)) |m + 1>,
  S^x = (S^+ + S^-) / 2,  S^y = (S^+ - S^-) / (2i).
The squeezing parameter is Eq. 15: with <S> along x (Eq. 13: <S^x> = (N/2) cos^(N-1)(chi t),
<S^y> = <S^z> = 0), xi^2 / N is the smallest eigenvalue of the y-z block of the second moments
<S^a S^b> (symmetrised) divided by <S^x>^2.
"""
from __future__ import annotations

import numpy as np
from scipy.special import gammaln


def dicke_spin_ops(n):
    """S^z, S^+, S^-, S^x, S^y of total spin S = n/2 in the basis m = -S..S (ascending)."""
    s = 0.5 * n
    m = np.arange(-s, s + 1.0)
    Sz = np.diag(m).astype(np.complex128)
    up = np.sqrt(s * (s + 1) - m[:-1] * (m[:-1] + 1))
    Sp = np.zeros((n + 1, n + 1), dtype=np.complex128)
    Sp[np.arange(1, n + 1), np.arange(n)] = up      # <m+1| S^+ |m>
    Sm = Sp.conj().T
    Sx = 0.5 * (Sp + Sm)
    Sy = -0.5j * (Sp - Sm)
    return Sz, Sp, Sm, Sx, Sy


def oat_state(n, t, chi=1.0):
    """Amplitudes over |S, m> (m ascending) of exp(-i chi t (S^z)^2) |+x>^n."""
    s = 0.5 * n
    m = np.arange(-s, s + 1.0)
    k = (m + s).astype(int)                          # number of up spins
    log_binom = gammaln(n + 1) - gammaln(k + 1) - gammaln(n - k + 1)
    c = np.exp(0.5 * log_binom - 0.5 * n * np.log(2.0))
    return c * np.exp(-1j * chi * t * m * m)


def oat_moments(n, t, chi=1.0):
    """<S^a> and <S^a S^b> (a, b in x, y, z) of the OAT state at time t."""
    Sz, _, _, Sx, Sy = dicke_spin_ops(n)
    v = oat_state(n, t, chi)
    ops = {"x": Sx, "y": Sy, "z": Sz}
    out = {a: complex(np.vdot(v, M @ v)) for a, M in ops.items()}
    for a, A in ops.items():
        for b, B in ops.items():
            out[a + b] = complex(np.vdot(v, A @ (B @ v)))
    return out


def squeezing_xi2(mom, n):
    """Eq. 15 from the moments: N (yy + zz - sqrt((yy - zz)^2 + (yz + zy)^2)) / (2 <S^x>^2),
    with the second moments real parts (yz + zy is real for a Hermitian pair)."""
    yy, zz = mom["yy"].real, mom["zz"].real
    yz = (mom["yz"] + mom["zy"]).real
    sx = mom["x"].real
    return n * (yy + zz - np.sqrt((yy - zz) ** 2 + yz ** 2)) / (2.0 * sx * sx)
