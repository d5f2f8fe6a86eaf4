// tll_poly.cuh -- generated by gen_poly.py (Remez, relative error).
// f(w) = w + (w^3) Q(w^2) with P = 1 + s Q(s); Q's coefficients,
// low order first (P's constant term is exactly 1).
#pragma once

// atan on [0.0, 1.0], degree 9 in w^2: max rel err 2.37e-09 (float64), 7.35e-08 (float32 Horner)
#define TLL_ATAN_NC 9
#define TLL_ATAN_COEFS {-3.333328366e-01f, 1.999826580e-01f, -1.426193267e-01f, 1.094203070e-01f, -8.377315104e-02f, 5.755210295e-02f, -3.080459684e-02f, 1.072694361e-02f, -1.753930119e-03f}

// atanh on [0.0, 0.5], degree 6 in w^2: max rel err 1.26e-09 (float64), 6.86e-08 (float32 Horner)
#define TLL_ATANH_NC 6
#define TLL_ATANH_COEFS {3.333328366e-01f, 2.000301927e-01f, 1.421579868e-01f, 1.187057048e-01f, 4.985036701e-02f, 1.785548776e-01f}

