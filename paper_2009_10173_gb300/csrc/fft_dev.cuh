// Shared-memory radix-2 FFT of interleaved complex lines and the 16-point
// twiddle constants, used by the lateral-FFT operator form and by the
// band-pass filter along time.
#pragma once

#include <cuda_runtime.h>

namespace oam {
namespace fftdev {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Twiddles w_j = exp(-2 pi i j / P), j < P/2, into shared memory.
__device__ __forceinline__ void load_twiddles(float2 *tw, int P) {
  for (int j = threadIdx.x; j < (P >> 1); j += blockDim.x) {
    float s, c;
    sincospif(-2.0f * (float)j / (float)P, &s, &c);
    tw[j] = make_float2(c, s);
  }
}

// In-place radix-2 decimation-in-time transforms of KC interleaved lines of
// P complex values (a[i * KC + c], loaded in bit-reversed order), sign -1
// (forward) or +1 (inverse, unscaled).  Two consecutive stages (spans h and
// 2h) act on the same four elements {i, i+h, i+2h, i+3h}, so a thread runs
// both in registers: one shared-memory pass per two stages (a leading single
// stage when log2 P is odd).
template <int KC>
__device__ void fft_lines(float2 *a, const float2 *tw, int P, int lgP, bool inverse) {
  __syncthreads();
  int half = 1;
  if (lgP & 1) {  // span-1 stage: twiddle 1
    for (int id = threadIdx.x; id < (P >> 1) * KC; id += blockDim.x) {
      const int c = id % KC, t = id / KC;
      const float2 x0 = a[(2 * t) * KC + c], x1 = a[(2 * t + 1) * KC + c];
      a[(2 * t) * KC + c] = make_float2(x0.x + x1.x, x0.y + x1.y);
      a[(2 * t + 1) * KC + c] = make_float2(x0.x - x1.x, x0.y - x1.y);
    }
    __syncthreads();
    half = 2;
  }
  const float sgn = inverse ? -1.0f : 1.0f;
  for (; half < P; half <<= 2) {
    const int s1 = P / (2 * half), s2 = P / (4 * half);  // twiddle strides of the two stages
    for (int id = threadIdx.x; id < (P >> 2) * KC; id += blockDim.x) {
      const int c = id % KC, t = id / KC;
      const int q = t & (half - 1);
      const int i0 = 4 * (t - q) + q;
      float2 x0 = a[i0 * KC + c], x1 = a[(i0 + half) * KC + c];
      float2 x2 = a[(i0 + 2 * half) * KC + c], x3 = a[(i0 + 3 * half) * KC + c];
      float2 w = tw[q * s1];
      w.y *= sgn;
      float2 y = cmul(x1, w);
      x1 = make_float2(x0.x - y.x, x0.y - y.y);
      x0 = make_float2(x0.x + y.x, x0.y + y.y);
      y = cmul(x3, w);
      x3 = make_float2(x2.x - y.x, x2.y - y.y);
      x2 = make_float2(x2.x + y.x, x2.y + y.y);
      float2 wa = tw[q * s2], wb = tw[(q + half) * s2];
      wa.y *= sgn;
      wb.y *= sgn;
      y = cmul(x2, wa);
      a[i0 * KC + c] = make_float2(x0.x + y.x, x0.y + y.y);
      a[(i0 + 2 * half) * KC + c] = make_float2(x0.x - y.x, x0.y - y.y);
      y = cmul(x3, wb);
      a[(i0 + half) * KC + c] = make_float2(x1.x + y.x, x1.y + y.y);
      a[(i0 + 3 * half) * KC + c] = make_float2(x1.x - y.x, x1.y - y.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int x, int lg) { return (int)(__brev((unsigned)x) >> (32 - lg)); }

constexpr float kRsqrt2 = 0.70710678118654752f;  // cos(pi/4) = sin(pi/4)
constexpr float kCosPi8 = 0.92387953251128676f;  // cos(pi/8)
constexpr float kSinPi8 = 0.38268343236508977f;  // sin(pi/8)

// W_N^u = exp(-2 pi i u / N) for N <= 16 (u < N/2), from the constants above.
__device__ __forceinline__ float2 w16(int N, int u) {
  switch (u * (16 / N)) {  // in sixteenths of a turn
    case 0: return make_float2(1.0f, 0.0f);
    case 1: return make_float2(kCosPi8, -kSinPi8);
    case 2: return make_float2(kRsqrt2, -kRsqrt2);
    case 3: return make_float2(kSinPi8, -kCosPi8);
    case 4: return make_float2(0.0f, -1.0f);
    case 5: return make_float2(-kSinPi8, -kCosPi8);
    case 6: return make_float2(-kRsqrt2, -kRsqrt2);
    default: return make_float2(-kCosPi8, -kSinPi8);  // 7
  }
}

}  // namespace fftdev
}  // namespace oam
