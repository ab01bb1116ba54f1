// Packed two-wide FP32 fused multiply-add (sm_100 and later): two independent FMAs in one
// instruction, each lane rounded exactly as fmaf.
#pragma once

#include <cuda_runtime.h>

namespace asd {

// (u, v) += (wc, ws) * g as one packed two-wide FP32 FMA (each lane rounds like fmaf).
__device__ __forceinline__ void fma2(float &u, float &v, float wc, float ws, float g)
{
    asm("{\n\t.reg .b64 pa, pb, pc;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %4};\n\t"
        "mov.b64 pc, {%0, %1};\n\t"
        "fma.rn.f32x2 pc, pa, pb, pc;\n\t"
        "mov.b64 {%0, %1}, pc;\n\t}"
        : "+f"(u), "+f"(v)
        : "f"(wc), "f"(ws), "f"(g));
}

}  // namespace asd
