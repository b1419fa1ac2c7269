// Small device helpers: typed loads/stores (BF16 storage with FP32 arithmetic) and
// precision-overloaded math.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace fn {

__device__ __forceinline__ double ld(const double* p) { return *p; }
__device__ __forceinline__ float ld(const float* p) { return *p; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st(double* p, double v) { *p = v; }
__device__ __forceinline__ void st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void st(double* p, float v) { *p = (double)v; }
__device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st(__nv_bfloat16* p, double v) { *p = __float2bfloat16_rn((float)v); }
// BF16 storage keeps the value slab (t = 0) of the stream activations as a pair: bf16(v)
// in the slab itself and the remainder bf16(v - bf16(v)) in an extra slab after the last
// tangent slab, about 16 significant bits together.  The tangent slabs keep one bf16.
template <typename Act> struct SplitValue { static constexpr bool value = false; };
template <> struct SplitValue<__nv_bfloat16> { static constexpr bool value = true; };
__device__ __forceinline__ float bf16_rem(float v) { return v - __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ void st_lo(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(bf16_rem(v)); }
__device__ __forceinline__ void st_lo(__nv_bfloat16* p, double v) {
  *p = __float2bfloat16_rn((float)(v - (double)__bfloat162float(__float2bfloat16_rn((float)v))));
}
template <typename T, typename V> __device__ __forceinline__ void st_lo(T*, V) {}

// Warp-level BF16 tensor-core product (m16n8k16, FP32 accumulation) and the hi/lo split of
// two FP32 values into packed BF16 pairs: bf16(v) and bf16(v - bf16(v)).
__device__ __forceinline__ void split_pack(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *(const uint32_t*)&h;
  lo = *(const uint32_t*)&l;
}

__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}


// two adjacent elements at an even element offset from an aligned base
__device__ __forceinline__ void st2(double* p, double a, double b) { *(double2*)p = make_double2(a, b); }
__device__ __forceinline__ void st2(float* p, float a, float b) { *(float2*)p = make_float2(a, b); }
__device__ __forceinline__ void st2(__nv_bfloat16* p, float a, float b) { *(__nv_bfloat162*)p = __floats2bfloat162_rn(a, b); }
__device__ __forceinline__ void st2_lo(__nv_bfloat16* p, float a, float b) {
  *(__nv_bfloat162*)p = __floats2bfloat162_rn(bf16_rem(a), bf16_rem(b));
}
template <typename T, typename V> __device__ __forceinline__ void st2_lo(T*, V, V) {}

__device__ __forceinline__ float f_tanh(float x) { return tanhf(x); }
__device__ __forceinline__ double f_tanh(double x) { return tanh(x); }
// tanh for the BF16-storage mode, whose activations are rounded to 8 mantissa bits:
// tanh x = 1 - 2 / (e^{2x} + 1) with the fast exponential and division intrinsics.  Its
// absolute error is a few 1e-7 (cancellation near x = 0 costs relative, not absolute,
// accuracy); e^{2x} overflowing to inf gives exactly 1, underflowing to 0 gives -1.
__device__ __forceinline__ float tanh_fast(float x) { return 1.0f - __fdividef(2.0f, __expf(2.0f * x) + 1.0f); }
template <typename Act> __device__ __forceinline__ float act_tanh(float x) {
  if constexpr (std::is_same<Act, __nv_bfloat16>::value) return tanh_fast(x);
  else return tanhf(x);
}
template <typename Act> __device__ __forceinline__ double act_tanh(double x) { return tanh(x); }
__device__ __forceinline__ float f_exp(float x) { return expf(x); }
__device__ __forceinline__ double f_exp(double x) { return exp(x); }
__device__ __forceinline__ float f_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double f_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float f_log(float x) { return logf(x); }
__device__ __forceinline__ double f_log(double x) { return log(x); }
__device__ __forceinline__ float f_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double f_abs(double x) { return fabs(x); }

// Row of electron i of walker w in the walker-aligned tile layout.
__device__ __forceinline__ int64_t tile_row(int w, int i, int N, int wpt) {
  const int q = w / wpt;
  return (int64_t)q * 128 + (int64_t)(w - q * wpt) * N + i;
}

}  // namespace fn
