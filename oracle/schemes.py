"""CFET coefficient tables, Legendre polynomials, Gauss-Legendre quadrature, g_{i,m}.

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

Everything here is transcribed from the paper independently of the CUDA
library's own host tables.  Citations use the paper's section numbers and
its equation / table labels.

Conventions
-----------
* ``f[i, n]`` holds f_{i+1, n+1} of the paper (0-based arrays, 1-based paper).
* A scheme is stored as its *half table*: the rows the paper prints.  The
  full s x nA table follows from rule (R1), Eq. (FSymm), Sec. 4.1:
  f_{s-i+1,n} = (-1)^{n+1} f_{i,n}; for odd s the central row carries odd n
  only.
* The number of Gauss-Legendre points M equals the number of Legendre terms
  A_1..A_M the scheme uses (Sec. 7: N/2+1 points for optimised schemes that
  include A_{N/2+1}; N/2 points for schemes built from A_1..A_{N/2} by rule
  (R2), e.g. CF4:2 in Eq. (UCF4Gauss) uses the two-point rule).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------
# Shifted Legendre polynomials on [0, 1]  (Sec. 3.1, recurrence before
# Eq. (PSymm))
# --------------------------------------------------------------------------
def legendre_shifted(n: int, x):
    """P_n(x) on [0,1] from the three-term recurrence of Sec. 3.1:
    P_0 = 1, P_1 = 2x - 1, P_{n+1} = ((2n+1)/(n+1)) (2x-1) P_n - (n/(n+1)) P_{n-1}.
    """
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if n == 0:
        return p_prev
    p = 2.0 * x - 1.0
    for k in range(1, n):
        p_next = ((2 * k + 1) / (k + 1)) * (2.0 * x - 1.0) * p - (k / (k + 1)) * p_prev
        p_prev, p = p, p_next
    return p


# --------------------------------------------------------------------------
# Gauss-Legendre points and weights on [0, 1]  (Sec. 7, Table tab:GaussLeg)
# --------------------------------------------------------------------------
def gauss_legendre(M: int):
    """Points x_m and weights w_m of M-point Gauss-Legendre quadrature on [0,1],
    written out from the closed forms of Table tab:GaussLeg (Sec. 7)."""
    if M == 1:
        x = [0.5]
        w = [1.0]
    elif M == 2:
        d = math.sqrt(3.0) / 6.0
        x = [0.5 - d, 0.5 + d]
        w = [0.5, 0.5]
    elif M == 3:
        d = math.sqrt(3.0 / 20.0)
        x = [0.5 - d, 0.5, 0.5 + d]
        w = [5.0 / 18.0, 4.0 / 9.0, 5.0 / 18.0]
    elif M == 4:
        r = 2.0 * math.sqrt(6.0 / 5.0)
        d_out = math.sqrt((3.0 + r) / 28.0)
        d_in = math.sqrt((3.0 - r) / 28.0)
        x = [0.5 - d_out, 0.5 - d_in, 0.5 + d_in, 0.5 + d_out]
        s30 = math.sqrt(30.0)
        w = [(18.0 - s30) / 72.0, (18.0 + s30) / 72.0, (18.0 + s30) / 72.0, (18.0 - s30) / 72.0]
    else:
        raise ValueError("the paper tabulates Gauss-Legendre rules for M = 1..4 only")
    return np.array(x, dtype=np.float64), np.array(w, dtype=np.float64)


# --------------------------------------------------------------------------
# Scheme tables (Sec. 4.2-4.4 and 5.2-5.3)
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Scheme:
    name: str
    order: int      # N
    s: int          # number of exponentials
    nA: int         # number of Legendre terms A_1..A_nA used (= GL points M)
    half: tuple     # printed rows: tuple of tuples, row i -> (f_{i,1}, ..., f_{i,nA})


def _cf64_f11() -> float:
    # CF6:4, Table 6thCFET (Sec. 4.3): closed form of f_{1,1}
    s6 = math.sqrt(6.0)
    return 0.5 + (5400.0 - 600.0 * s6) ** (1.0 / 3.0) / 60.0 + ((9.0 + s6) / 5.0) ** (1.0 / 3.0) / (2.0 * 3.0 ** (2.0 / 3.0))


def _make_tables():
    T = {}
    # CF2:1, midpoint rule Eq. (UCF2): s = 1, f_{1,1} = 1
    T["CF2:1"] = Scheme("CF2:1", 2, 1, 1, ((1.0,),))
    # CF4:2, Table 4thCFET / Eq. (UCF4:2): f11 = 1/2, f12 = 1/3 (s = 2)
    T["CF4:2"] = Scheme("CF4:2", 4, 2, 2, ((0.5, 1.0 / 3.0),))
    # CF4:3, Table 4thCFET: f11 = 11/40, f12 = 20/87, central f21 = 9/20
    T["CF4:3"] = Scheme("CF4:3", 4, 3, 2, ((11.0 / 40.0, 20.0 / 87.0), (9.0 / 20.0, 0.0)))
    # CF4:3Opt, Table 4thCFETOpt / Eq. (CF4Optimal)
    T["CF4:3Opt"] = Scheme("CF4:3Opt", 4, 3, 3,
                           ((11.0 / 40.0, 20.0 / 87.0, 7.0 / 50.0), (9.0 / 20.0, 0.0, -7.0 / 25.0)))
    # CF6:4, Table 6thCFET: closed forms; the central rows vanish, leaving
    # four exponentials (rows 1, 2 and their mirror images).
    f11 = _cf64_f11()
    f12 = f11 - (2.0 / 3.0) * f11 * f11
    f13 = 1.0 / (10.0 - 10.0 * f11)
    f21 = 0.5 - f11
    f22 = (1.0 - 4.0 * f11 + 2.0 * f11 * f11) / 3.0
    f23 = -f13
    T["CF6:4"] = Scheme("CF6:4", 6, 4, 3, ((f11, f12, f13), (f21, f22, f23)))

    def five(name, nA, r1, r2):
        # s = 5 tables of Sec. 4.3 / 5.3: f31 = 1 - 2 f21 - 2 f11, f32 = 0,
        # f33 = -2 f23 - 2 f13, f34 = 0 (central row, odd n only)
        mid = [1.0 - 2.0 * r2[0] - 2.0 * r1[0], 0.0, -2.0 * r2[2] - 2.0 * r1[2]]
        if nA == 4:
            mid.append(0.0)
        return Scheme(name, 6, 5, nA, (tuple(r1), tuple(r2), tuple(mid)))

    # CF6:5, Table 6thCFET
    T["CF6:5"] = five("CF6:5", 3,
                      (0.16, 0.14587456942714338561, 0.11762370828143015682),
                      (0.38752405202531186588, 0.15089113704380764664, -0.12805075909013044594))
    # CF6:5b, Table 6thCFET (f_{2,2} printed with 16 digits; used as printed)
    T["CF6:5b"] = five("CF6:5b", 3,
                       (0.2, 0.1746879190177786220, 0.12406375705333586606),
                       (0.34815492558797391479, 0.1068765450953683, -0.139021313323765096675))
    # CF6:5Imp, Table 6thCFETOpt
    T["CF6:5Imp"] = five("CF6:5Imp", 4,
                         (0.16, 0.14587456942714338561, 0.11762370828143015682, 0.074),
                         (0.38752405202531186588, 0.15089113704380764664, -0.12805075909013044594,
                          -0.212530296697694739551))
    # CF6:5Opt, Table 6thCFETOpt
    T["CF6:5Opt"] = five("CF6:5Opt", 4,
                         (0.1714, 0.15409059414309687213, 0.11947178242929061641, 0.07195),
                         (0.37496374319946236513, 0.13813675394387646682, -0.13090674649282935743,
                          -0.21123356253315514306))
    # CF6:6, Table 6thCFET (s = 6: f31 = 1/2 - f11 - f21, f33 = -f13 - f23)
    r1 = (0.16, 0.15101538937746543493, 0.13304616813239630479)
    r2 = (-0.22738164742696330169, -0.087654259755115431662, 0.069919836812656575583)
    r3 = (0.5 - r1[0] - r2[0], 0.21035154512209824847, -r1[2] - r2[2])
    T["CF6:6"] = Scheme("CF6:6", 6, 6, 3, (r1, r2, r3))
    # CF6:6Opt, Table 6thCFETOpt
    r1 = (0.3952, 0.35629343479227292880, 0.27848030437681878641, 0.1579)
    r2 = (-0.22432144875476807927, -0.19935407393749030416, -0.15625650102884866893, -0.09512)
    r3 = (0.5 - r1[0] - r2[0], 0.1145, -r1[2] - r2[2], -0.16475168057141371958)
    T["CF6:6Opt"] = Scheme("CF6:6Opt", 6, 6, 4, (r1, r2, r3))
    # CF8:11, Table 8thCoeff: rows 1..5 with n = 1..4, central row 6 with
    # odd n only (f_{6,1}, f_{6,3}).
    T["CF8:11"] = Scheme("CF8:11", 8, 11, 4, (
        (0.169715531043933180094151, 0.152866146944615909929839,
         0.119167378745981369601216, 0.068619226448029559107538),
        (0.379420807516005431504230, 0.148839980923180990943008,
         -0.115880829186628075021088, -0.188555246668412628269760),
        (0.469459306644050573017994, -0.379844237839363505173921,
         0.022898814729462898505141, 0.571855043580130805495594),
        (-0.448225927391070886302766, 0.362889857410989942809900,
         -0.022565582830528472333301, -0.544507517141613383517695),
        (-0.293924473106317605373923, -0.026255628265819381983204,
         0.096761509131620390100068, 0.000018330145571671744069),
        (0.447109510586798614120629, 0.0, -0.200762581179816221704073, 0.0),
    ))
    return T


SCHEMES = _make_tables()

# Default scheme per order: CF2:1; CF4:2 (two exponentials, two GL nodes);
# CF6:5Opt (recommended in Sec. 12); CF8:11 (the only 8th-order table).
DEFAULT_FOR_ORDER = {2: "CF2:1", 4: "CF4:2", 6: "CF6:5Opt", 8: "CF8:11"}


def full_table(scheme: Scheme) -> np.ndarray:
    """Expand the printed half table into the full s x nA array by rule (R1),
    Eq. (FSymm): f_{s-i+1,n} = (-1)^{n+1} f_{i,n}."""
    s, nA = scheme.s, scheme.nA
    f = np.zeros((s, nA), dtype=np.float64)
    for i, row in enumerate(scheme.half):          # i is 0-based: paper row i+1
        for n0, val in enumerate(row):             # n0 is 0-based: paper n = n0+1
            f[i, n0] = val
            mirror = s - 1 - i                     # paper row s - (i+1) + 1
            sign = (-1.0) ** ((n0 + 1) + 1)
            if mirror != i:
                f[mirror, n0] = sign * val
    if s % 2 == 1:
        c = s // 2
        for n0 in range(nA):
            if (n0 + 1) % 2 == 0 and f[c, n0] != 0.0:
                raise ValueError("central exponential must carry odd n only (R1)")
    return f


def g_coefficients(scheme: Scheme):
    """g_{i,m} = w_m sum_{n=1}^{nA} (2n-1) P_{n-1}(x_m) f_{i,n}  (Sec. 7, after
    Eq. (OmGLeg)), with M = nA Gauss-Legendre points.

    Returns (g [s x M], x [M], w [M], f [s x nA]).
    """
    f = full_table(scheme)
    M = scheme.nA
    x, w = gauss_legendre(M)
    g = np.zeros((scheme.s, M), dtype=np.float64)
    for i in range(scheme.s):
        for m in range(M):
            acc = 0.0
            for n in range(1, scheme.nA + 1):
                acc += (2 * n - 1) * legendre_shifted(n - 1, x[m]) * f[i, n - 1]
            g[i, m] = w[m] * acc
    return g, x, w, f


def get(name_or_order) -> Scheme:
    if isinstance(name_or_order, int):
        return SCHEMES[DEFAULT_FOR_ORDER[name_or_order]]
    return SCHEMES[name_or_order]
