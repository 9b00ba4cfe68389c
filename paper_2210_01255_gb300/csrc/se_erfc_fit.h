// Generated by gen_erfc_fit.py: erfc(x) = exp(-x^2) t R(t), t = 1 / (1 + a x),
// R(t) = sum_k c_k t^k (Chebyshev interpolation of erfcx(x) / t on t in [0, 1]).
// max relative error of the polynomial (exact arithmetic): 8.70e-09
#pragma once
#define SE_ERFC_FIT_A 0.4
#define SE_ERFC_FIT_DEG 10
#define SE_ERFC_FIT_C0 0.22567583145616354
#define SE_ERFC_FIT_C1 0.2256763169273171
#define SE_ERFC_FIT_C2 0.20760072039863167
#define SE_ERFC_FIT_C3 0.17189057190002874
#define SE_ERFC_FIT_C4 0.11809512310530651
#define SE_ERFC_FIT_C5 0.08712064134251166
#define SE_ERFC_FIT_C6 -0.053793165709245604
#define SE_ERFC_FIT_C7 0.1468032448634684
#define SE_ERFC_FIT_C8 -0.24304173118280767
#define SE_ERFC_FIT_C9 0.14384106898691543
#define SE_ERFC_FIT_C10 -0.029868628431269858
