// Rounding helpers of the tensor-core kernels' split operands: an FP32 value v
// is carried as a 16-bit hi part and a 16-bit lo part (v = hi + lo + e), FP16
// with a power-of-two range scale or BF16 (FP32's range, fewer bits).
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

// Two floats rounded to BF16 and packed, v0 in the low half.
__device__ __forceinline__ uint32_t bf16x2_rn(float v0, float v1) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v1), "f"(v0));
    return d;
}

// Two floats rounded to FP16 and packed, v0 in the low half; and the FP16 values back.
__device__ __forceinline__ uint32_t f16x2_rn(float v0, float v1) {
    uint32_t d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v1), "f"(v0));
    return d;
}
__device__ __forceinline__ float f16_lo(uint32_t h) { return __half2float(__ushort_as_half((unsigned short)(h & 0xffffu))); }
__device__ __forceinline__ float f16_hi(uint32_t h) { return __half2float(__ushort_as_half((unsigned short)(h >> 16))); }

// The power of two 2^k with m 2^k in [2^13, 2^14) (1 for m = 0 or not finite), with k at
// most 64: a largest |value| below 2^-50 is scaled by 2^64 only, so that the scales and
// their products stay finite (such values then sit below 2^13 and lose FP16 precision).
__host__ __device__ inline float f16_range_scale(float m) {
    if (!(m > 0.0f) || !isfinite(m)) return 1.0f;
    int e;
    frexpf(m, &e);   // m = f 2^e, f in [0.5, 1)
    return ldexpf(1.0f, 14 - e < 64 ? 14 - e : 64);
}
