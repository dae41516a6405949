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
// A-lines to global memory.  Each sample is read from and written to HBM once
// and goes through shared memory four times each way at NF = 2048.
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
  int NF = 0, lgNF = 0, KC = 0;  // transform size, its log2, complex lines per block
  float *d_hb = nullptr;     // [NF] spectrum of the taps over NF, in bit-reversed order
  float *d_stage = nullptr;  // signal-sized staging buffer: F s ahead of the adjoint
  size_t bytes = 0;          // device bytes of the two buffers
};

}  // namespace oam

namespace {

using namespace oam::fftdev;

constexpr int kFirThreads = 256;
constexpr int kFirMaxSize = 8192;  // largest transform: 65 KB of shared memory per line pair

size_t fir_smem(int NF, int KC) { return sizeof(float2) * ((size_t)KC * NF + NF / 8); }

// Shared-memory layout of KC interleaved complex lines: point i of line c at
// i*KC + c, plus one pad slot after every 8 points so that the 8-point groups
// of the middle pass, read with the group index fastest, spread over all banks.
template <int KC>
__device__ __forceinline__ int slot(int i, int c) { return i * KC + c + (i >> 3); }

constexpr float kRsqrt2 = 0.70710678118654752f;  // cos(pi/4) = sin(pi/4)
constexpr float kCos8 = 0.92387953251128676f;    // cos(pi/8)
constexpr float kSin8 = 0.38268343236508977f;    // sin(pi/8)

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// W_N^u = exp(-2 pi i u / N) for N <= 16 (u < N/2), from the constants above.
__device__ __forceinline__ float2 w_small(int N, int u) {
  const int e = u * (16 / N);  // in sixteenths
  switch (e) {
    case 0: return make_float2(1.0f, 0.0f);
    case 1: return make_float2(kCos8, -kSin8);
    case 2: return make_float2(kRsqrt2, -kRsqrt2);
    case 3: return make_float2(kSin8, -kCos8);
    case 4: return make_float2(0.0f, -1.0f);
    case 5: return make_float2(-kSin8, -kCos8);
    case 6: return make_float2(-kRsqrt2, -kRsqrt2);
    default: return make_float2(-kCos8, -kSin8);  // 7
  }
}

// One shared-memory pass of R = 2^r decimation-in-frequency stages with spans
// 2^(k+r-1) down to 2^k, in registers, for point group (c, q, blk): the
// points i0 + m 2^k, i0 = blk 2^(k+r) + q, q < 2^k.  Span S = 2^(k+j) maps
// (u, w) at (p, p + S) to (u + w, (u - w) W_2S^(p mod S)) with
// p mod S = q + (m mod 2^j) 2^k, so its twiddle is W_2S^q W_2^(j+1)^(m mod 2^j):
// the first factor is b^(2^(r-1-j)) for b = W_2^(k+r)^q (one sincospif, then
// squarings), the second a constant.  Loads come from global memory (points at
// or beyond nt read as zero) when kFromGlobal, else from shared memory.
template <int KC, int r, bool kFromGlobal>
__device__ __forceinline__ void dif_pass(float2 *a, int NF, int k, const float *x, long long line0, long long n_lines,
                                         int nt) {
  constexpr int R = 1 << r;
  const int groups = NF >> r;
  for (int id = threadIdx.x; id < groups * KC; id += blockDim.x) {
    const int c = id % KC, t = id / KC;
    const int q = t & ((1 << k) - 1), blk = t >> k;
    const int i0 = (blk << (k + r)) | q;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int n = i0 + (m << k);
      if (kFromGlobal) {
        const long long l0 = line0 + 2 * c, l1 = l0 + 1;
        float re = 0.0f, im = 0.0f;
        if (n < nt) {
          if (l0 < n_lines) re = x[l0 * nt + n];
          if (l1 < n_lines) im = x[l1 * nt + n];
        }
        v[m] = make_float2(re, im);
      } else {
        v[m] = a[slot<KC>(n, c)];
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
        const float2 u = v[m], w = v[m + S];
        v[m] = cadd(u, w);
        const int um = m & (S - 1);
        const float2 tw = um == 0 ? pw[j] : cmul(pw[j], w_small(2 * S, um));
        v[m + S] = cmul(csub(u, w), tw);
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) a[slot<KC>(i0 + (m << k), c)] = v[m];
  }
}

// The matching decimation-in-time inverse pass (spans 2^k up to 2^(k+r-1)):
// (u, w) at (p, p + S) go to (u + w conj(W), u - w conj(W)), W as above.
// Results go to global memory (points below nt only) when kToGlobal, else
// back to shared memory.
template <int KC, int r, bool kToGlobal>
__device__ __forceinline__ void dit_pass(float2 *a, int NF, int k, float *y, long long line0, long long n_lines,
                                         int nt) {
  constexpr int R = 1 << r;
  const int groups = NF >> r;
  for (int id = threadIdx.x; id < groups * KC; id += blockDim.x) {
    const int c = id % KC, t = id / KC;
    const int q = t & ((1 << k) - 1), blk = t >> k;
    const int i0 = (blk << (k + r)) | q;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = a[slot<KC>(i0 + (m << k), c)];
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
        const float2 tw = um == 0 ? pw[j] : cmul(pw[j], w_small(2 * S, um));
        const float2 u = v[m], w = cmul(v[m + S], cconj(tw));
        v[m] = cadd(u, w);
        v[m + S] = csub(u, w);
      }
    }
    if (kToGlobal) {
      const long long l0 = line0 + 2 * c, l1 = l0 + 1;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int n = i0 + (m << k);
        if (n < nt) {
          if (l0 < n_lines) y[l0 * nt + n] = v[m].x;
          if (l1 < n_lines) y[l1 * nt + n] = v[m].y;
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) a[slot<KC>(i0 + (m << k), c)] = v[m];
    }
  }
}

// The middle of the convolution for one 8-point group g of line c, in
// registers: forward stages of spans 4, 2, 1 (the group then holds spectrum
// entries in bit-reversed order), the product with the filter's spectrum in
// the same order, inverse stages of spans 1, 2, 4.
template <int KC>
__device__ __forceinline__ void mid_group(float2 *a, int g, int c, const float4 *__restrict__ hb4) {
  float2 v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = a[slot<KC>(8 * g + j, c)];
  // forward span 4: W_8^j = (1, (1-i)/sqrt2, -i, (-1-i)/sqrt2)
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 u = v[j], w = v[j + 4];
    v[j] = make_float2(u.x + w.x, u.y + w.y);
    const float2 d = make_float2(u.x - w.x, u.y - w.y);
    if (j == 0) v[4] = d;
    if (j == 1) v[5] = make_float2(kRsqrt2 * (d.x + d.y), kRsqrt2 * (d.y - d.x));
    if (j == 2) v[6] = make_float2(d.y, -d.x);
    if (j == 3) v[7] = make_float2(kRsqrt2 * (d.y - d.x), -kRsqrt2 * (d.x + d.y));
  }
  // forward span 2: W_4^j = (1, -i)
#pragma unroll
  for (int b = 0; b < 8; b += 4) {
    const float2 u0 = v[b], w0 = v[b + 2], u1 = v[b + 1], w1 = v[b + 3];
    v[b] = make_float2(u0.x + w0.x, u0.y + w0.y);
    v[b + 2] = make_float2(u0.x - w0.x, u0.y - w0.y);
    v[b + 1] = make_float2(u1.x + w1.x, u1.y + w1.y);
    v[b + 3] = make_float2(u1.y - w1.y, w1.x - u1.x);
  }
  // forward span 1, product, inverse span 1
  const float4 h0 = hb4[2 * g], h1 = hb4[2 * g + 1];
  const float hs[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
  for (int b = 0; b < 8; b += 2) {
    const float2 u = v[b], w = v[b + 1];
    const float2 p = make_float2((u.x + w.x) * hs[b], (u.y + w.y) * hs[b]);
    const float2 m = make_float2((u.x - w.x) * hs[b + 1], (u.y - w.y) * hs[b + 1]);
    v[b] = make_float2(p.x + m.x, p.y + m.y);
    v[b + 1] = make_float2(p.x - m.x, p.y - m.y);
  }
  // inverse span 2: conj W_4^j = (1, i)
#pragma unroll
  for (int b = 0; b < 8; b += 4) {
    const float2 u0 = v[b], w0 = v[b + 2], u1 = v[b + 1];
    const float2 w1 = make_float2(-v[b + 3].y, v[b + 3].x);
    v[b] = make_float2(u0.x + w0.x, u0.y + w0.y);
    v[b + 2] = make_float2(u0.x - w0.x, u0.y - w0.y);
    v[b + 1] = make_float2(u1.x + w1.x, u1.y + w1.y);
    v[b + 3] = make_float2(u1.x - w1.x, u1.y - w1.y);
  }
  // inverse span 4: conj W_8^j = (1, (1+i)/sqrt2, i, (-1+i)/sqrt2)
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 u = v[j], x = v[j + 4];
    float2 w = x;
    if (j == 1) w = make_float2(kRsqrt2 * (x.x - x.y), kRsqrt2 * (x.x + x.y));
    if (j == 2) w = make_float2(-x.y, x.x);
    if (j == 3) w = make_float2(-kRsqrt2 * (x.x + x.y), kRsqrt2 * (x.x - x.y));
    v[j] = make_float2(u.x + w.x, u.y + w.y);
    v[j + 4] = make_float2(u.x - w.x, u.y - w.y);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) a[slot<KC>(8 * g + j, c)] = v[j];
}

// First forward pass (from global memory) and last inverse pass (to global
// memory) with r0 = ((log2 NF - 3) mod 4, or 4) stages at k = log2 NF - r0.
template <int KC, bool kForward>
__device__ __forceinline__ void edge_pass(int r0, float2 *a, int NF, int k, const float *x, float *y, long long line0,
                                          long long n_lines, int nt) {
  switch (r0) {
    case 1:
      if (kForward) dif_pass<KC, 1, true>(a, NF, k, x, line0, n_lines, nt);
      else dit_pass<KC, 1, true>(a, NF, k, y, line0, n_lines, nt);
      break;
    case 2:
      if (kForward) dif_pass<KC, 2, true>(a, NF, k, x, line0, n_lines, nt);
      else dit_pass<KC, 2, true>(a, NF, k, y, line0, n_lines, nt);
      break;
    case 3:
      if (kForward) dif_pass<KC, 3, true>(a, NF, k, x, line0, n_lines, nt);
      else dit_pass<KC, 3, true>(a, NF, k, y, line0, n_lines, nt);
      break;
    default:
      if (kForward) dif_pass<KC, 4, true>(a, NF, k, x, line0, n_lines, nt);
      else dit_pass<KC, 4, true>(a, NF, k, y, line0, n_lines, nt);
      break;
  }
}

// y = F x for n_lines A-lines of nt samples (x and y may alias: a block reads
// all of its lines before it writes any).  Block b holds real lines
// 2 KC b .. 2 KC b + 2 KC - 1; complex line c carries real lines 2c (real
// part) and 2c + 1 (imaginary part).  NF >= 16.  hb: the filter's spectrum
// over NF, in bit-reversed order (NF floats, 16-byte aligned).  Forward
// stages: spans NF/2 .. 2^k0 straight from global memory, then passes of four
// down to span 8, then the register middle (spans 4, 2, 1, the product and
// back); the inverse mirrors them and its last pass writes to global memory.
template <int KC>
__global__ void __launch_bounds__(kFirThreads) k_fir_lines(const float *x, float *y, long long n_lines, int nt,
                                                           int NF, int lgNF, const float *__restrict__ hb) {
  extern __shared__ float2 a[];
  const long long line0 = (long long)blockIdx.x * (2 * KC);
  const int r0 = ((lgNF - 3) & 3) ? ((lgNF - 3) & 3) : 4;
  const int k0 = lgNF - r0;
  edge_pass<KC, true>(r0, a, NF, k0, x, nullptr, line0, n_lines, nt);
  __syncthreads();
  for (int k = k0 - 4; k >= 3; k -= 4) {
    dif_pass<KC, 4, false>(a, NF, k, nullptr, 0, 0, 0);
    __syncthreads();
  }
  const int groups = NF >> 3;
  for (int id = threadIdx.x; id < groups * KC; id += blockDim.x)
    mid_group<KC>(a, id % groups, id / groups, reinterpret_cast<const float4 *>(hb));
  __syncthreads();
  for (int k = 3; k + 4 <= k0; k += 4) {
    dit_pass<KC, 4, false>(a, NF, k, nullptr, 0, 0, 0);
    __syncthreads();
  }
  edge_pass<KC, false>(r0, a, NF, k0, nullptr, y, line0, n_lines, nt);
}

oam_status set_smem(const void *fn, size_t bytes) {
  if (bytes > 48 * 1024)
    OAM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return OAM_OK;
}

template <int KC>
oam_status launch_fir(const FirLayout *F, const float *x, float *y, long long n_lines, int nt, cudaStream_t st) {
  const size_t smem = fir_smem(F->NF, KC);
  oam_status rc = set_smem((const void *)k_fir_lines<KC>, smem);
  if (rc) return rc;
  const long long blocks = (n_lines + 2 * KC - 1) / (2 * KC);
  if (blocks <= 0) return OAM_OK;
  k_fir_lines<KC><<<(unsigned)blocks, kFirThreads, smem, st>>>(x, y, n_lines, nt, F->NF, F->lgNF, F->d_hb);
  OAM_LAUNCHED();
  return OAM_OK;
}

// Complex lines per block: about 64 KB of lines in shared memory.
int fir_lines_per_block(int NF) { return std::max(1, std::min(16, 8192 / NF)); }

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
  switch (F->KC) {
    case 16: return launch_fir<16>(F, x, y, lines, m->grid.nt, st);
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
  F->KC = fir_lines_per_block(NF);
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
  OAM_CUDA_TRY(cudaStreamSynchronize(st));
  return OAM_OK;
}

oam_status oam_filter_signals(const oam_model *m, const float *d_in, float *d_out, void *stream) {
  if (!m || !d_in || !d_out || !m->fir) return OAM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 15) return OAM_ERR_INVALID_ARG;
  return fir_apply(m, d_in, d_out, as_stream(stream));
}

}  // extern "C"
