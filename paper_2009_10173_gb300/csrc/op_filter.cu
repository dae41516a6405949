// Band-pass filtering along time, and the filtered operators F A and A^T F.
//
// Results: before inversion the raw signals and the model matrix are band-pass
// filtered (0.5-80 MHz in the second simulation, 1-120 MHz in vivo).  The
// filter F here is a zero-phase FIR with 2L + 1 even taps h[-L..L], applied to
// every A-line of nt samples with zeros outside [0, nt) and the centred nt
// outputs kept; oam_bandpass_taps designs one by the Blackman-windowed sinc
// method.  Filtering every slab column S[b][a][k][:] with F gives the operator
// F A (the filter acts along time, A laterally and over depth, so the two
// commute), and its adjoint is A^T F because F is symmetric.  A model with a
// filter therefore applies F after its forward operator and before its
// adjoint; the slab stays unfiltered and banded (a filter sharp enough for a
// 0.5 MHz cut-off at 250 MS/s is about as long as the A-line and would widen
// every band to all of it).
//
// On the device F is a circular convolution of length NF, a power of two with
// NF >= nt + min(L, nt - 1), so no wrap reaches [0, nt).  Each pair of A-lines
// is one complex line (real and imaginary parts), transformed by a radix-2
// decimation-in-frequency FFT (natural order in, bit-reversed order out),
// multiplied by the filter's spectrum (real because the taps are even,
// pre-scaled by 1/NF, stored in bit-reversed order) and transformed back by a
// decimation-in-time inverse FFT (bit-reversed in, natural order out), so no
// permutation pass is needed.  Stages run in registers, up to four per pass
// over shared memory: the first forward pass reads the A-lines from global
// memory, the three smallest spans of both transforms and the product share
// one pass on 8-point groups, and the last inverse pass writes the filtered
// A-lines to global memory.  A thread carries the same points of two complex
// lines as packed FP32 pairs, so each twiddle serves both.  Each sample is read
// from and written to HBM once and goes through shared memory four times each
// way at NF = 2048.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "fft_dev.cuh"
#include "internal.cuh"

using namespace oam;

namespace oam {

struct FirLayout {
  int L = 0;                 // half length as set (taps with |m| >= nt never reach the output)
  int NF = 0, lgNF = 0, KP = 0;  // transform size, its log2, complex line pairs per block
  float *d_hb = nullptr;     // [NF] spectrum of the taps over NF, in bit-reversed order
  float *d_stage = nullptr;  // signal-sized staging buffer: F s ahead of the adjoint
  size_t bytes = 0;          // device bytes of the two buffers
};

}  // namespace oam

namespace {

using namespace oam::fftdev;

constexpr int kFirThreads = 256;
constexpr int kFirMaxSize = 8192;  // largest transform: 144 KiB of shared memory for one line pair

size_t fir_smem(int NF, int KP) { return sizeof(ulonglong2) * ((size_t)KP * NF + NF / 8); }

// Packed FP32 pairs (two lanes of one 64-bit register) and their arithmetic.
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {  // a b + c
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ uint64_t f2_splat(float v) { return f2_pack(v, v); }
__device__ __forceinline__ float2 f2_unpack(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

// The same point of two complex lines c and c + 1: re = (re_c, re_c+1),
// im = (im_c, im_c+1).  Every operation below acts on both lines at once.
struct Cx2 {
  uint64_t re, im;
};
__device__ __forceinline__ Cx2 x_add(Cx2 a, Cx2 b) { return Cx2{f2_add(a.re, b.re), f2_add(a.im, b.im)}; }
__device__ __forceinline__ Cx2 x_sub(Cx2 a, Cx2 b) { return Cx2{f2_sub(a.re, b.re), f2_sub(a.im, b.im)}; }
// a w for one complex w shared by both lines
__device__ __forceinline__ Cx2 x_mul(Cx2 a, float2 w) {
  const uint64_t wr = f2_splat(w.x), wi = f2_splat(w.y), nwi = f2_splat(-w.y);
  return Cx2{f2_fma(a.re, wr, f2_mul(a.im, nwi)), f2_fma(a.im, wr, f2_mul(a.re, wi))};
}

// Shared-memory layout: one 16-byte slot per (point i, line pair p) holding
// (re_c, re_c+1, im_c, im_c+1), at i*KP + p, plus one pad slot after every 8
// points, so that 8-point groups read with the group index fastest land in
// distinct bank groups.  Points 2^k apart (2^k >= 8) are (KP << k) + 2^(k-3)
// slots apart.
template <int KP>
__device__ __forceinline__ int slot(int i, int p) { return i * KP + p + (i >> 3); }

// One shared-memory pass of R = 2^r decimation-in-frequency stages with spans
// 2^(k+r-1) down to 2^k, in registers, for point group (p, q, blk): the
// points i0 + m 2^k, i0 = blk 2^(k+r) + q, q < 2^k, of line pair p.  Span
// S = 2^(k+j) maps (u, w) at (n, n + S) to (u + w, (u - w) W_2S^(n mod S)) with
// n mod S = q + (m mod 2^j) 2^k, so its twiddle is W_2S^q W_2^(j+1)^(m mod 2^j):
// the first factor is b^(2^(r-1-j)) for b = W_2^(k+r)^q (one sincospif, then
// squarings), the second a constant.  With kFromGlobal the points come from
// the A-lines in global memory (points at or beyond nt, and lines at or beyond
// n_lines, read as zero): line pair p is real lines line0 + 4p .. line0 + 4p + 3
// as (re_c, im_c, re_c+1, im_c+1).
template <int KP, int r, bool kFromGlobal>
__device__ __forceinline__ void dif_pass(ulonglong2 *a, int NF, int k, const float *x, long long line0,
                                         long long n_lines, int nt) {
  constexpr int R = 1 << r;
  const int groups = NF >> r;
  const int ds = (KP << k) + (1 << (k - 3));
  for (int id = threadIdx.x; id < groups * KP; id += blockDim.x) {
    const int p = id % KP, t = id / KP;
    const int q = t & ((1 << k) - 1), blk = t >> k;
    const int i0 = (blk << (k + r)) | q;
    const int s0 = slot<KP>(i0, p);
    Cx2 v[R];
    if (kFromGlobal) {
      const long long lb = line0 + 4 * p;
      const bool ok0 = lb < n_lines, ok1 = lb + 1 < n_lines, ok2 = lb + 2 < n_lines, ok3 = lb + 3 < n_lines;
      const long long base = lb * nt + i0;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int n = i0 + (m << k);
        float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, e3 = 0.0f;
        if (n < nt) {
          const long long o = base + (m << k);
          if (ok0) e0 = x[o];
          if (ok1) e1 = x[o + nt];
          if (ok2) e2 = x[o + 2 * (long long)nt];
          if (ok3) e3 = x[o + 3 * (long long)nt];
        }
        v[m] = Cx2{f2_pack(e0, e2), f2_pack(e1, e3)};
      }
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const ulonglong2 u = a[s0 + m * ds];
        v[m] = Cx2{u.x, u.y};
      }
    }
    float2 pw[r];  // pw[j] = W_2^(k+j+1)^q
    sincospif(-2.0f * (float)q / (float)(1 << (k + r)), &pw[r - 1].y, &pw[r - 1].x);
#pragma unroll
    for (int j = r - 2; j >= 0; --j) pw[j] = cmul(pw[j + 1], pw[j + 1]);
#pragma unroll
    for (int j = r - 1; j >= 0; --j) {
      const int S = 1 << j;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (m & S) continue;
        const Cx2 u = v[m], w = v[m + S];
        v[m] = x_add(u, w);
        const int um = m & (S - 1);
        const float2 tw = um == 0 ? pw[j] : cmul(pw[j], w16(2 * S, um));
        v[m + S] = x_mul(x_sub(u, w), tw);
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) a[s0 + m * ds] = make_ulonglong2(v[m].re, v[m].im);
  }
}

// The matching decimation-in-time inverse pass (spans 2^k up to 2^(k+r-1)):
// (u, w) at (n, n + S) go to (u + w conj(W), u - w conj(W)), W as above.  With
// kToGlobal the results go to the A-lines in global memory (points below nt
// and lines below n_lines only), else back to shared memory.
template <int KP, int r, bool kToGlobal>
__device__ __forceinline__ void dit_pass(ulonglong2 *a, int NF, int k, float *y, long long line0, long long n_lines,
                                         int nt) {
  constexpr int R = 1 << r;
  const int groups = NF >> r;
  const int ds = (KP << k) + (1 << (k - 3));
  for (int id = threadIdx.x; id < groups * KP; id += blockDim.x) {
    const int p = id % KP, t = id / KP;
    const int q = t & ((1 << k) - 1), blk = t >> k;
    const int i0 = (blk << (k + r)) | q;
    const int s0 = slot<KP>(i0, p);
    Cx2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const ulonglong2 u = a[s0 + m * ds];
      v[m] = Cx2{u.x, u.y};
    }
    float2 pw[r];
    sincospif(-2.0f * (float)q / (float)(1 << (k + r)), &pw[r - 1].y, &pw[r - 1].x);
#pragma unroll
    for (int j = r - 2; j >= 0; --j) pw[j] = cmul(pw[j + 1], pw[j + 1]);
#pragma unroll
    for (int j = 0; j < r; ++j) {
      const int S = 1 << j;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (m & S) continue;
        const int um = m & (S - 1);
        const float2 tw = um == 0 ? pw[j] : cmul(pw[j], w16(2 * S, um));
        const Cx2 u = v[m], w = x_mul(v[m + S], make_float2(tw.x, -tw.y));
        v[m] = x_add(u, w);
        v[m + S] = x_sub(u, w);
      }
    }
    if (kToGlobal) {
      const long long lb = line0 + 4 * p;
      const bool ok0 = lb < n_lines, ok1 = lb + 1 < n_lines, ok2 = lb + 2 < n_lines, ok3 = lb + 3 < n_lines;
      const long long base = lb * nt + i0;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int n = i0 + (m << k);
        if (n < nt) {
          const long long o = base + (m << k);
          const float2 re = f2_unpack(v[m].re), im = f2_unpack(v[m].im);
          if (ok0) y[o] = re.x;
          if (ok1) y[o + nt] = im.x;
          if (ok2) y[o + 2 * (long long)nt] = re.y;
          if (ok3) y[o + 3 * (long long)nt] = im.y;
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) a[s0 + m * ds] = make_ulonglong2(v[m].re, v[m].im);
    }
  }
}

// The middle of the convolution for one 8-point group g of line pair p, in
// registers: forward stages of spans 4, 2, 1 (the group then holds spectrum
// entries in bit-reversed order), the product with the filter's spectrum in
// the same order, inverse stages of spans 1, 2, 4.  Products with +-i are
// folded into the additions.
template <int KP>
__device__ __forceinline__ void mid_group(ulonglong2 *a, int g, int p, const float4 *__restrict__ hb4) {
  const int base = slot<KP>(8 * g, p);
  Cx2 v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const ulonglong2 u = a[base + j * KP];
    v[j] = Cx2{u.x, u.y};
  }
  const uint64_t R2 = f2_splat(kRsqrt2), NR2 = f2_splat(-kRsqrt2);
  // forward span 4: W_8^j = (1, (1-i)/sqrt2, -i, (-1-i)/sqrt2)
  {
    const Cx2 u0 = v[0], w0 = v[4], u1 = v[1], w1 = v[5], u2 = v[2], w2 = v[6], u3 = v[3], w3 = v[7];
    v[0] = x_add(u0, w0);
    v[4] = x_sub(u0, w0);
    v[1] = x_add(u1, w1);
    const Cx2 d1 = x_sub(u1, w1);
    v[5] = Cx2{f2_mul(R2, f2_add(d1.re, d1.im)), f2_mul(R2, f2_sub(d1.im, d1.re))};
    v[2] = x_add(u2, w2);
    v[6] = Cx2{f2_sub(u2.im, w2.im), f2_sub(w2.re, u2.re)};
    v[3] = x_add(u3, w3);
    const Cx2 d3 = x_sub(u3, w3);
    v[7] = Cx2{f2_mul(R2, f2_sub(d3.im, d3.re)), f2_mul(NR2, f2_add(d3.re, d3.im))};
  }
  // forward span 2: W_4^j = (1, -i)
#pragma unroll
  for (int b = 0; b < 8; b += 4) {
    const Cx2 u0 = v[b], w0 = v[b + 2], u1 = v[b + 1], w1 = v[b + 3];
    v[b] = x_add(u0, w0);
    v[b + 2] = x_sub(u0, w0);
    v[b + 1] = x_add(u1, w1);
    v[b + 3] = Cx2{f2_sub(u1.im, w1.im), f2_sub(w1.re, u1.re)};
  }
  // forward span 1, product, inverse span 1
  const float4 h0 = hb4[2 * g], h1 = hb4[2 * g + 1];
  const float hs[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
  for (int b = 0; b < 8; b += 2) {
    const uint64_t ha = f2_splat(hs[b]), hc = f2_splat(hs[b + 1]);
    const Cx2 u = v[b], w = v[b + 1];
    const Cx2 P = Cx2{f2_mul(f2_add(u.re, w.re), ha), f2_mul(f2_add(u.im, w.im), ha)};
    const Cx2 M = Cx2{f2_mul(f2_sub(u.re, w.re), hc), f2_mul(f2_sub(u.im, w.im), hc)};
    v[b] = x_add(P, M);
    v[b + 1] = x_sub(P, M);
  }
  // inverse span 2: conj W_4^j = (1, i); w i = (-w.im, w.re)
#pragma unroll
  for (int b = 0; b < 8; b += 4) {
    const Cx2 u0 = v[b], w0 = v[b + 2], u1 = v[b + 1], w1 = v[b + 3];
    v[b] = x_add(u0, w0);
    v[b + 2] = x_sub(u0, w0);
    v[b + 1] = Cx2{f2_sub(u1.re, w1.im), f2_add(u1.im, w1.re)};
    v[b + 3] = Cx2{f2_add(u1.re, w1.im), f2_sub(u1.im, w1.re)};
  }
  // inverse span 4: conj W_8^j = (1, (1+i)/sqrt2, i, (-1+i)/sqrt2)
  {
    const Cx2 u0 = v[0], x0 = v[4], u1 = v[1], x1 = v[5], u2 = v[2], x2 = v[6], u3 = v[3], x3 = v[7];
    v[0] = x_add(u0, x0);
    v[4] = x_sub(u0, x0);
    const uint64_t d1 = f2_sub(x1.re, x1.im), s1 = f2_add(x1.re, x1.im);  // x1 conj W_8 = r (d1, s1)
    v[1] = Cx2{f2_fma(R2, d1, u1.re), f2_fma(R2, s1, u1.im)};
    v[5] = Cx2{f2_fma(NR2, d1, u1.re), f2_fma(NR2, s1, u1.im)};
    v[2] = Cx2{f2_sub(u2.re, x2.im), f2_add(u2.im, x2.re)};
    v[6] = Cx2{f2_add(u2.re, x2.im), f2_sub(u2.im, x2.re)};
    const uint64_t s3 = f2_add(x3.re, x3.im), d3 = f2_sub(x3.re, x3.im);  // x3 conj W_8^3 = r (-s3, d3)
    v[3] = Cx2{f2_fma(NR2, s3, u3.re), f2_fma(R2, d3, u3.im)};
    v[7] = Cx2{f2_fma(R2, s3, u3.re), f2_fma(NR2, d3, u3.im)};
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) a[base + j * KP] = make_ulonglong2(v[j].re, v[j].im);
}

// First forward pass (from global memory) and last inverse pass (to global
// memory) with r0 = ((log2 NF - 3) mod 4, or 4) stages at k = log2 NF - r0.
template <int KP, bool kForward>
__device__ __forceinline__ void edge_pass(int r0, ulonglong2 *a, int NF, int k, const float *x, float *y,
                                          long long line0, long long n_lines, int nt) {
  switch (r0) {
    case 1:
      if (kForward) dif_pass<KP, 1, true>(a, NF, k, x, line0, n_lines, nt);
      else dit_pass<KP, 1, true>(a, NF, k, y, line0, n_lines, nt);
      break;
    case 2:
      if (kForward) dif_pass<KP, 2, true>(a, NF, k, x, line0, n_lines, nt);
      else dit_pass<KP, 2, true>(a, NF, k, y, line0, n_lines, nt);
      break;
    case 3:
      if (kForward) dif_pass<KP, 3, true>(a, NF, k, x, line0, n_lines, nt);
      else dit_pass<KP, 3, true>(a, NF, k, y, line0, n_lines, nt);
      break;
    default:
      if (kForward) dif_pass<KP, 4, true>(a, NF, k, x, line0, n_lines, nt);
      else dit_pass<KP, 4, true>(a, NF, k, y, line0, n_lines, nt);
      break;
  }
}

// y = F x for n_lines A-lines of nt samples (x and y may alias: a block reads
// all of its lines before it writes any).  Block b holds real lines
// 4 KP b .. 4 KP b + 4 KP - 1 as 2 KP complex lines (real and imaginary part
// from consecutive real lines), processed in line pairs.  NF >= 16.  hb: the
// filter's spectrum over NF, in bit-reversed order (NF floats, 16-byte
// aligned).  Forward stages: spans NF/2 .. 2^k0 straight from global memory,
// then passes of four down to span 8, then the register middle (spans 4, 2, 1,
// the product and back); the inverse mirrors them and its last pass writes to
// global memory.
template <int KP>
__global__ void __launch_bounds__(kFirThreads, 2) k_fir_lines(const float *x, float *y, long long n_lines, int nt,
                                                              int NF, int lgNF, const float *__restrict__ hb) {
  extern __shared__ ulonglong2 a[];
  const long long line0 = (long long)blockIdx.x * (4 * KP);
  const int r0 = ((lgNF - 3) & 3) ? ((lgNF - 3) & 3) : 4;
  const int k0 = lgNF - r0;
  edge_pass<KP, true>(r0, a, NF, k0, x, nullptr, line0, n_lines, nt);
  __syncthreads();
  for (int k = k0 - 4; k >= 3; k -= 4) {
    dif_pass<KP, 4, false>(a, NF, k, nullptr, 0, 0, 0);
    __syncthreads();
  }
  const int groups = NF >> 3;
  for (int id = threadIdx.x; id < groups * KP; id += blockDim.x)
    mid_group<KP>(a, id % groups, id / groups, reinterpret_cast<const float4 *>(hb));
  __syncthreads();
  for (int k = 3; k + 4 <= k0; k += 4) {
    dit_pass<KP, 4, false>(a, NF, k, nullptr, 0, 0, 0);
    __syncthreads();
  }
  edge_pass<KP, false>(r0, a, NF, k0, nullptr, y, line0, n_lines, nt);
}

oam_status set_smem(const void *fn, size_t bytes) {
  if (bytes > 48 * 1024)
    OAM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return OAM_OK;
}

template <int KP>
oam_status launch_fir(const FirLayout *F, const float *x, float *y, long long n_lines, int nt, cudaStream_t st) {
  const size_t smem = fir_smem(F->NF, KP);
  oam_status rc = set_smem((const void *)k_fir_lines<KP>, smem);
  if (rc) return rc;
  const long long blocks = (n_lines + 4 * KP - 1) / (4 * KP);
  if (blocks <= 0) return OAM_OK;
  k_fir_lines<KP><<<(unsigned)blocks, kFirThreads, smem, st>>>(x, y, n_lines, nt, F->NF, F->lgNF, F->d_hb);
  OAM_LAUNCHED();
  return OAM_OK;
}

// Line pairs per block: about 64 KB of points in shared memory.
int fir_pairs_per_block(int NF) { return std::max(1, std::min(8, 4096 / NF)); }

double sinc(double x) { return x == 0.0 ? 1.0 : std::sin(M_PI * x) / (M_PI * x); }

}  // namespace

void oam::fir_free(oam_model *m, cudaStream_t st) {
  FirLayout *F = m->fir;
  if (!F) return;
  if (F->d_hb) cudaFreeAsync(F->d_hb, st);
  if (F->d_stage) cudaFreeAsync(F->d_stage, st);
  m->bytes -= F->bytes;
  delete F;
  m->fir = nullptr;
}

oam_status oam::fir_apply(const oam_model *m, const float *x, float *y, cudaStream_t st) {
  const FirLayout *F = m->fir;
  if (!F) return OAM_ERR_INVALID_ARG;
  const long long lines = (long long)m->grid.py * m->grid.px;
  switch (F->KP) {
    case 8: return launch_fir<8>(F, x, y, lines, m->grid.nt, st);
    case 4: return launch_fir<4>(F, x, y, lines, m->grid.nt, st);
    case 2: return launch_fir<2>(F, x, y, lines, m->grid.nt, st);
    case 1: return launch_fir<1>(F, x, y, lines, m->grid.nt, st);
  }
  return OAM_ERR_DEVICE;
}

float *oam::fir_stage(const oam_model *m) { return m->fir ? m->fir->d_stage : nullptr; }
int oam::fir_half_len(const oam_model *m) { return m->fir ? m->fir->L : -1; }
int oam::fir_size(const oam_model *m) { return m->fir ? m->fir->NF : 0; }

extern "C" {

oam_status oam_bandpass_taps(double f_lo_hz, double f_hi_hz, double fs_hz, int32_t half_len, double *taps) {
  if (!taps || !(fs_hz > 0) || !std::isfinite(fs_hz)) return OAM_ERR_INVALID_ARG;
  if (!(f_lo_hz >= 0) || !(f_lo_hz < f_hi_hz) || !(f_hi_hz <= fs_hz / 2)) return OAM_ERR_INVALID_ARG;
  if (half_len < 0 || half_len > OAM_MAX_FIR_HALF) return OAM_ERR_INVALID_ARG;
  const double L1 = half_len + 1.0;
  for (int m = 0; m <= half_len; ++m) {
    const double window = 0.42 + 0.5 * std::cos(M_PI * m / L1) + 0.08 * std::cos(2.0 * M_PI * m / L1);
    const double ideal = 2.0 * f_hi_hz / fs_hz * sinc(2.0 * f_hi_hz * m / fs_hz) -
                         2.0 * f_lo_hz / fs_hz * sinc(2.0 * f_lo_hz * m / fs_hz);
    taps[m] = window * ideal;
  }
  return OAM_OK;
}

oam_status oam_model_set_filter(oam_model *m, const double *taps, int32_t half_len, void *stream) {
  if (!m) return OAM_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  if (!taps || half_len < 0) {  // remove
    if (m->fir) ++m->generation;
    fir_free(m, st);
    OAM_CUDA_TRY(cudaStreamSynchronize(st));
    return OAM_OK;
  }
  if (half_len > OAM_MAX_FIR_HALF) return OAM_ERR_INVALID_ARG;
  for (int i = 0; i <= half_len; ++i)
    if (!std::isfinite(taps[i])) return OAM_ERR_INVALID_ARG;
  const int nt = m->grid.nt;
  const int Le = std::min(half_len, nt - 1);  // taps that can reach [0, nt)
  int NF = 16, lg = 4;  // at least one outer stage on each side of the 8-point middle
  while (NF < nt + Le) {
    NF <<= 1;
    ++lg;
  }
  if (NF > kFirMaxSize) return OAM_ERR_INVALID_ARG;
  // spectrum of the even taps on NF points (real): h0 + 2 sum_m h_m cos(2 pi f m / NF),
  // over NF, stored at the bit reversal of f (the order the forward transform leaves)
  std::vector<double> ct(NF);
  for (int j = 0; j < NF; ++j) ct[j] = std::cos(2.0 * M_PI * j / NF);
  std::vector<float> hh(NF);
  for (int f = 0; f < NF; ++f) {
    double acc = 0.0;
    for (int k = Le; k >= 1; --k) acc += taps[k] * ct[(size_t)((long long)f * k % NF)];
    int r = 0;
    for (int b = 0; b < lg; ++b) r |= ((f >> b) & 1) << (lg - 1 - b);
    hh[r] = (float)((taps[0] + 2.0 * acc) / NF);
  }
  FirLayout *F = new (std::nothrow) FirLayout();
  if (!F) return OAM_ERR_OOM;
  F->L = half_len;
  F->NF = NF;
  F->lgNF = lg;
  F->KP = fir_pairs_per_block(NF);
  const size_t hbytes = sizeof(float) * hh.size(), sbytes = sizeof(float) * sig_elems(m);
  if (cudaMallocAsync((void **)&F->d_hb, hbytes, st) != cudaSuccess ||
      cudaMallocAsync((void **)&F->d_stage, sbytes, st) != cudaSuccess) {
    cudaGetLastError();
    if (F->d_hb) cudaFreeAsync(F->d_hb, st);
    if (F->d_stage) cudaFreeAsync(F->d_stage, st);
    cudaStreamSynchronize(st);
    delete F;
    return OAM_ERR_OOM;
  }
  F->bytes = hbytes + sbytes;
  if (cudaMemcpyAsync(F->d_hb, hh.data(), hbytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaFreeAsync(F->d_hb, st);
    cudaFreeAsync(F->d_stage, st);
    cudaStreamSynchronize(st);
    delete F;
    return OAM_ERR_CUDA;
  }
  fir_free(m, st);
  m->fir = F;
  m->bytes += F->bytes;
  ++m->generation;
  OAM_CUDA_TRY(cudaStreamSynchronize(st));
  return OAM_OK;
}

oam_status oam_filter_signals(const oam_model *m, const float *d_in, float *d_out, void *stream) {
  if (!m || !d_in || !d_out || !m->fir) return OAM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 15) return OAM_ERR_INVALID_ARG;
  return fir_apply(m, d_in, d_out, as_stream(stream));
}

}  // extern "C"
