// sincos_poly.cuh -- written by gen_sincos_poly.py (do not edit): sine and
// cosine of a full turn on the FP32 FMA pipe, s in [-1/2, 1/2]:
//   sin(2 pi s) = s (S0 + S1 u + ... + S5 u^5),  cos(2 pi s) = C0 + C1 u + ... + C6 u^6,  u = s^2
// (near-minimax fits by Lawson's reweighted least squares, rounded to float).
#pragma once

#define RSI_POLY_S0 6.283182621e+00f
#define RSI_POLY_S1 -4.134142303e+01f
#define RSI_POLY_S2 8.159619141e+01f
#define RSI_POLY_S3 -7.658014679e+01f
#define RSI_POLY_S4 4.120560074e+01f
#define RSI_POLY_S5 -1.227158928e+01f
#define RSI_POLY_C0 1.000000000e+00f
#define RSI_POLY_C1 -1.973920441e+01f
#define RSI_POLY_C2 6.493911743e+01f
#define RSI_POLY_C3 -8.545016479e+01f
#define RSI_POLY_C4 6.016785812e+01f
#define RSI_POLY_C5 -2.596841049e+01f
#define RSI_POLY_C6 6.529749870e+00f
