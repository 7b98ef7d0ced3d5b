// Paired FP32 arithmetic (PTX fma.rn.f32x2, sm_100 and later): two IEEE fused multiply-adds with one instruction,
// each lane rounded exactly as fmaf rounds it, so results are bit-identical to the scalar form.
#pragma once

#include <cstdint>

namespace rascal {

__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(uint64_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// (a.lo * b.lo + c.lo, a.hi * b.hi + c.hi)
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

}  // namespace rascal
