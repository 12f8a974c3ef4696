// Per-row epilogue math shared by the CUDA-core and tensor-core forward kernels.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include "dae_internal.h"

namespace dae {

struct ActD { float s0, s1, s2, s3; };

// act and its first three derivatives at a (tanh, sin or identity).
// For tanh, 1 - t^2 loses relative accuracy as |t| -> 1, so for |t| >= 1/2 the
// derivative is formed as 4e/(1+e)^2 with e = exp(-2|a|) (= sech^2 a).
__device__ __forceinline__ ActD act_d(int act, float a) {
    ActD d;
    if (act == DAE_ACT_TANH) {
        float t = tanhf(a);
        float t2 = t * t;
        float s1;
        if (t2 < 0.25f) {
            s1 = 1.0f - t2;
        } else {
            float e = expf(-2.0f * fabsf(a));
            float den = 1.0f + e;
            s1 = 4.0f * e / (den * den);
        }
        d.s0 = t;
        d.s1 = s1;
        d.s2 = -2.0f * t * s1;
        d.s3 = -2.0f * s1 * (1.0f - 3.0f * t2);
    } else if (act == DAE_ACT_SIN) {
        float sn, cs;
        sincosf(a, &sn, &cs);
        d.s0 = sn; d.s1 = cs; d.s2 = -sn; d.s3 = -cs;
    } else {
        d.s0 = a; d.s1 = 1.0f; d.s2 = 0.0f; d.s3 = 0.0f;
    }
    return d;
}

// Multicomplex activation of the stacked components (Sec. 4.1 Eq. 16, Sec. 4.3).
// For x = a + b i1 + c (i2 + i3) + d (i1i2 + i1i3) + g i2i3 + h i1i2i3 with b, c ~ h_cs,
// d, g ~ h_cs^2, h ~ h_cs^3, the multicomplex Taylor expansion of act(x) gives each
// component to leading order in h_cs; the terms of higher order in h_cs that the
// paper discards (Sec. 4.4: "high-order terms of h is discarded") are dropped, so
// the components are exact up to O(h_cs^2) relative and rounding:
//   i2 : s1 c               i2i3 : s1 g + s2 c^2
//   i1 : s1 b               i1i2 : s1 d + s2 b c
//   i1i2i3 : s1 h + s2 (b g + 2 c d) + s3 b c^2
__device__ __forceinline__ void mc_shared(const ActD& D, float c, float gw, float g0,
                                          float& oc, float& ogw, float& og0) {
    float s2cc = D.s2 * c * c;
    oc = D.s1 * c;
    ogw = fmaf(D.s1, gw, s2cc);
    og0 = fmaf(D.s1, g0, s2cc);
}

__device__ __forceinline__ void mc_group(const ActD& D, float c, float gw, float b, float dd,
                                         float hh, float& ob, float& od, float& oh) {
    ob = D.s1 * b;
    od = fmaf(D.s1, dd, D.s2 * b * c);
    oh = fmaf(D.s1, hh, fmaf(D.s2, fmaf(b, gw, 2.0f * c * dd), D.s3 * b * c * c));
}

// FP32 value rounded to the nearest TF32 value (10 explicit mantissa bits, ties away
// from zero), returned as an FP32 bit pattern.  The tf32 tensor-core path reads the
// low 13 mantissa bits as zero, so rounding here replaces a biased truncation.
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return __uint_as_float(y);
}

// out_bf16: 0 FP32 only, 1 FP32 + BF16 hi, 2 FP32 + BF16 hi + lo, kStoreTF32 FP32
// rounded to TF32 (the operand of the tf32 tensor-core GEMMs).

__device__ __forceinline__ void store_act(float v, float* Y, __nv_bfloat16* Yh,
                                          __nv_bfloat16* Yl, size_t idx, int out_bf16) {
    if (out_bf16 == kStoreTF32) {
        Y[idx] = tf32_rna(v);
        return;
    }
    Y[idx] = v;
    if (out_bf16) {
        __nv_bfloat16 hi = __float2bfloat16_rn(v);
        Yh[idx] = hi;
        if (out_bf16 == 2) Yl[idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

}  // namespace dae
