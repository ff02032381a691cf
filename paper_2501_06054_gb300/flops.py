"""Nominal algorithmic FLOP counts of one neutron history (FMA = 2 FLOP).

These are the floating-point operations the method needs per quadrature
term in FP32, counted from the formulas with software sin and cos (a
two-part reduction and two polynomials) and excluding integer work
(Philox, pixel arithmetic, selects). The table is fixed: it converts
histories/s into an equivalent FLOP/s for the roofline against the FP32
CUDA-core peak. Where a kernel takes sin and cos from the special-function
unit instead (the FP32 core-shell node loop), it executes fewer FP32
operations than counted here for the same terms.

  sphere amplitude g(Q r) = (sin x - x cos x) / x^3           33
      x, 1/x (2 mul), quadrant (FMA, add), 2-part reduction (2 FMA),
      r^2, sin poly (2 FMA), cos poly (3 FMA), r^3 (mul), sin r, cos r
      (2 FMA), the two quadrant forms (2 FMA), / x^3 (3 mul), S - C (add)
      (the factor 3 of f = 3 g is folded into the tables)
  cylinder radial factor 2 J1(Q r)/(Q r), x <= 8 product form  26
      x^2 = |Q x c|^2 r^2 (mul), zero factors (2 FMA), polynomial
      (8 FMA), product (2 mul), a^2 (mul), weighted sum (FMA)
  orientation node overhead (cylinder, ellipsoid)              60
      Q.c, |Q x c|^2 (11 FMA/mul), sqrt, 1/x, rsqrt (3), sinc (~26),
      weight products (3), Kahan (4)
  ellipsoid term: |Q|_eff^2 (FMA), rsqrt, x (mul), amplitude
                  without its own x, 1/x, g^2, weighted sum        2+1+1+31+1+2 = 38
  sphere node: amplitude, g^2, weighted sum                       33 + 3
  core-shell node: inner amplitude 33; outer amplitude by angle
      addition from the inner reduced angle: x, 1/x (2 mul), sin and
      cos of (r + q t) (2 mul + 2 FMA), two quadrant forms (2 FMA),
      / x^3 (3 mul), x^2 and its Taylor form (mul + 4 FMA) = 24;
      combination (mul, FMA, FMA) 5                                33 + 24 + 5
      per history sin, cos of q t                                   20
  frame node overhead (3-axis models): Q.A, Q.B, Q.C times the
      sizes (9 FMA/mul), weight and Kahan (5)                      20
  triaxial ellipsoid term: scale (mul), amplitude 33, g^2 and the
      weighted sum (2)                                             36
  parallelepiped term: three scaled arguments (3 mul), three sincs
      (3 x 20: reduction, sin polynomial, 1/y), product, square and
      weighted sum (3)                                             66
  capped cylinder and barbell: per cap slice (cos from the special-
      function unit, not counted): argument s Q_C z (mul), x^2 (mul),
      2 J1(x)/x for x <= 4 (6 FMA), c cos (mul), weighted sum (FMA)    17
      per radius node: s Q_C, |y| L/2 (2 mul), sinc (~20), cylinder
      amplitude (mul), x^2 (mul), 2 J1(x)/x (6 FMA) and its product
      (mul), F^2 and the weighted sum (3)                          40
      per orientation node as for the cylinder                     60
  shelled cylinders (core-shell, hollow, bicelle): per radius node
      two radial factors 2 J1(x)/x without their square and sum
      (2 x 23), the two sinc combinations (2 x (mul, FMA)), the
      amplitude (FMA), F^2 and the sum (FMA)                       56
      per orientation node: the cylinder's plus a second sinc      86
  core-shell ellipsoid: per radius node two ellipsoid terms without
      their square and sum (2 x 35), combination (mul, FMA), F^2
      and the sum (FMA)                                            75
      per orientation node as for the ellipsoid                    60
  per history: geometry (wavelength, pinholes, slab, detector
               point, Q, solid angle)                           150
               Percus-Yevick S(Q)                               40
"""

AMP = 33
CYL_TERM = 26
FRAME_NODE = 20
TRI_TERM = 36
BOX_TERM = 66
CS_NODE = 62
CS_HISTORY = 20
ORIENT_NODE = 60
GEOMETRY = 150
PY = 40
CAP_SLICE = 17
CAP_NODE = 40
CS_CYL_TERM = 56
CS_CYL_ORIENT = 86
CS_ELL_TERM = 75


def flops_per_history(kind: int, n_poly: int, n_orient: int = 1, sq: bool = False, n_cap: int = 16) -> int:
    if kind == 0:        # sphere
        per = n_poly * (AMP + 3)
    elif kind == 1:      # core-shell
        per = n_poly * CS_NODE + CS_HISTORY
    elif kind == 2:      # cylinder
        per = n_orient * (ORIENT_NODE + n_poly * CYL_TERM)
    elif kind == 4:      # triaxial ellipsoid (n_orient = frames)
        per = n_orient * (FRAME_NODE + n_poly * TRI_TERM)
    elif kind == 5:      # parallelepiped
        per = n_orient * (FRAME_NODE + n_poly * BOX_TERM)
    elif kind in (6, 7):  # capped cylinder, barbell
        per = n_orient * (ORIENT_NODE + n_poly * (CAP_NODE + n_cap * CAP_SLICE))
    elif kind in (8, 9, 11):  # core-shell cylinder, hollow cylinder, core-shell bicelle
        per = n_orient * (CS_CYL_ORIENT + n_poly * CS_CYL_TERM)
    elif kind == 10:     # core-shell ellipsoid
        per = n_orient * (ORIENT_NODE + n_poly * CS_ELL_TERM)
    else:                # ellipsoid
        per = n_orient * (ORIENT_NODE + n_poly * (AMP + 5))
    return per + GEOMETRY + (PY if sq else 0)


def fp32_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
