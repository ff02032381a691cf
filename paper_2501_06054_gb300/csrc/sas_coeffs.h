/* Generated by gen_coeffs.py -- FP32 coefficients of the device special
 * functions (own fits, see the generator's docstring). Do not edit. */
#pragma once

#define SAS_J1_X1 4.0f
/* fit errors (FP64): small 1.118e-10, modulus 3.425e-09, phase 1.404e-08, S 2.137e-08, C 9.145e-10 */
#define SAS_PIO2_1 1.570796371e+00f
#define SAS_PIO2_2 -4.371138829e-08f
#define SAS_PIO4_1 7.853981853e-01f
#define SAS_PIO4_2 -2.185569414e-08f
/* 2 J1(x)/x = (1 - s z1)(1 - s z2) h(s), s = x^2 <= 64; fit error of h 6.653e-10 */
#define SAS_J1P_SMAX 6.400000000e+01f
#define SAS_J1P_Z1 6.811074783e-02f
#define SAS_J1P_Z2 2.031758155e-02f
#define SAS_J1P_C_N 9
#define SAS_J1P_C {9.999999993e-01f, -3.657166892e-02f, 5.905152050e-04f, -5.678942625e-06f, 3.695457932e-08f, -1.747459127e-10f, 6.223534422e-13f, -1.621063721e-15f, 2.424090863e-18f}
/* 2 J1(x)/x = (1 - s z1)(1 - s z2)(1 - s z3) g(2 s / 144 - 1), s <= 144; fit error of g 2.165e-10 */
#define SAS_J1Q_SMAX 1.440000000e+02f
#define SAS_J1Q_Z1 6.811074783e-02f
#define SAS_J1Q_Z2 2.031758155e-02f
#define SAS_J1Q_Z3 9.661886729e-03f
#define SAS_J1Q_C_N 11
#define SAS_J1Q_C {1.169814826e-01f, -2.826843847e-01f, 2.994814183e-01f, -1.884617908e-01f, 8.024855756e-02f, -2.491085858e-02f, 5.920458534e-03f, -1.115097382e-03f, 1.711073644e-04f, -2.243371898e-05f, 2.410184778e-06f}
/* 2 J1(x)/x = r(s), s = x^2 <= 16; fit error 7.874e-09 */
#define SAS_J1R_SMAX 1.600000000e+01f
#define SAS_J1R_C_N 7
#define SAS_J1R_C {9.999999921e-01f, -1.249999514e-01f, 5.208284287e-03f, -1.084883597e-04f, 1.352971110e-06f, -1.098744745e-08f, 5.233149538e-11f}
/* 2 J1(x)/x = v(2 s / 36 - 1), s = x^2 <= 36; fit error 5.705e-08 */
#define SAS_J1V_SMAX 3.600000000e+01f
#define SAS_J1V_C_N 8
#define SAS_J1V_C {-7.217181136e-02f, -2.981637351e-01f, 4.605520289e-01f, -2.369276485e-01f, 6.421195081e-02f, -1.091158982e-02f, 1.293798204e-03f, -1.110028616e-04f}
/* sin r = r + r^3 S(r^2), cos r = 1 + r^2 C(r^2) */
#define SAS_SIN_C_N 3
#define SAS_SIN_C {-1.666666455e-01f, 8.332725399e-03f, -1.958295501e-04f}
#define SAS_COS_C_N 4
#define SAS_COS_C {-4.999999992e-01f, 4.166663354e-02f, -1.388677625e-03f, 2.437042503e-05f}
#define SAS_J1S_C_N 8
#define SAS_J1S_C {9.999999999e-01f, -1.999999986e+00f, 1.333333029e+00f, -4.444419945e-01f, 8.887918082e-02f, -1.183089002e-02f, 1.103495466e-03f, -6.449931052e-05f}
#define SAS_J1M_C_N 6
#define SAS_J1M_C {1.000000003e+00f, 1.171846577e-02f, -7.514159251e-04f, 1.757710064e-04f, -5.899622254e-05f, 1.244681187e-05f}
#define SAS_J1H_C_N 6
#define SAS_J1H_C {3.749999861e-01f, -1.025273366e-02f, 1.432409031e-03f, -4.877704056e-04f, 1.948607847e-04f, -4.437957135e-05f}
