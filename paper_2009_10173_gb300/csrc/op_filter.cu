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
// is one complex line (real and imaginary parts), transformed in shared memory
// by a radix-2 decimation-in-frequency FFT (natural order in, bit-reversed
// order out), multiplied by the filter's spectrum (real because the taps are
// even, pre-scaled by 1/NF, stored in bit-reversed order) and transformed back
// by a decimation-in-time inverse FFT (bit-reversed in, natural order out), so
// no permutation pass is needed.  The three smallest spans of both transforms
// and the product run in registers on 8-point groups; the other stages go two
// per shared-memory pass.  Each sample is read from and written to HBM once.
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
constexpr int kFirMaxSize = 8192;  // largest transform: 96 KB of shared memory (twiddles, one line pair)

size_t fir_smem(int NF, int KC) { return sizeof(float2) * ((size_t)NF / 2 + (size_t)KC * NF + NF / 8); }

// Shared-memory layout of KC interleaved complex lines: point i of line c at
// i*KC + c, plus one pad slot after every 8 points so that the 8-point groups
// of the middle pass, read with the group index fastest, spread over all banks.
template <int KC>
__device__ __forceinline__ int slot(int i, int c) { return i * KC + c + (i >> 3); }

constexpr float kRsqrt2 = 0.70710678118654752f;  // cos(pi/4) = sin(pi/4)

// The outer decimation-in-frequency stages (spans P/2 down to 8; sign -1):
// span s maps (u, w) at (j, j + s) of each block of 2s to (u + w, (u - w) W_2s^j).
// Two stages per shared-memory pass (spans 2h and h act on {i, i+h, i+2h, i+3h});
// a leading single stage when their count log2 P - 3 is odd.
template <int KC>
__device__ void dif_outer(float2 *a, const float2 *tw, int P, int lgP) {
  int h;
  if ((lgP - 3) & 1) {
    const int s = P >> 1;
    for (int id = threadIdx.x; id < s * KC; id += blockDim.x) {
      const int c = id % KC, j = id / KC;
      const float2 u = a[slot<KC>(j, c)], w = a[slot<KC>(j + s, c)];
      a[slot<KC>(j, c)] = make_float2(u.x + w.x, u.y + w.y);
      a[slot<KC>(j + s, c)] = cmul(make_float2(u.x - w.x, u.y - w.y), tw[j]);
    }
    __syncthreads();
    h = P >> 3;
  } else {
    h = P >> 2;
  }
  for (; h >= 8; h >>= 2) {
    const int s1 = P / (4 * h), s2 = P / (2 * h);  // W_4h^j = tw[j s1], W_2h^j = tw[j s2]
    for (int id = threadIdx.x; id < (P >> 2) * KC; id += blockDim.x) {
      const int c = id % KC, t = id / KC;
      const int q = t & (h - 1);
      const int i0 = 4 * (t - q) + q;
      const float2 x0 = a[slot<KC>(i0, c)], x1 = a[slot<KC>(i0 + h, c)];
      const float2 x2 = a[slot<KC>(i0 + 2 * h, c)], x3 = a[slot<KC>(i0 + 3 * h, c)];
      const float2 y0 = make_float2(x0.x + x2.x, x0.y + x2.y);
      const float2 y2 = cmul(make_float2(x0.x - x2.x, x0.y - x2.y), tw[q * s1]);
      const float2 y1 = make_float2(x1.x + x3.x, x1.y + x3.y);
      const float2 y3 = cmul(make_float2(x1.x - x3.x, x1.y - x3.y), tw[(q + h) * s1]);
      const float2 w = tw[q * s2];
      a[slot<KC>(i0, c)] = make_float2(y0.x + y1.x, y0.y + y1.y);
      a[slot<KC>(i0 + h, c)] = cmul(make_float2(y0.x - y1.x, y0.y - y1.y), w);
      a[slot<KC>(i0 + 2 * h, c)] = make_float2(y2.x + y3.x, y2.y + y3.y);
      a[slot<KC>(i0 + 3 * h, c)] = cmul(make_float2(y2.x - y3.x, y2.y - y3.y), w);
    }
    __syncthreads();
  }
}

// The outer decimation-in-time inverse stages (spans 8 up to P/2; sign +1):
// span s maps (u, w) at (j, j + s) to (u + w conj(W_2s^j), u - w conj(W_2s^j)).
// Two stages per pass (spans h and 2h), a trailing single stage when their
// count is odd.
template <int KC>
__device__ void dit_outer(float2 *a, const float2 *tw, int P, int lgP) {
  int h = 8;
  for (; 4 * h <= P; h <<= 2) {
    const int s1 = P / (2 * h), s2 = P / (4 * h);  // W_2h^j = tw[j s1], W_4h^j = tw[j s2]
    for (int id = threadIdx.x; id < (P >> 2) * KC; id += blockDim.x) {
      const int c = id % KC, t = id / KC;
      const int q = t & (h - 1);
      const int i0 = 4 * (t - q) + q;
      float2 x0 = a[slot<KC>(i0, c)], x1 = a[slot<KC>(i0 + h, c)];
      float2 x2 = a[slot<KC>(i0 + 2 * h, c)], x3 = a[slot<KC>(i0 + 3 * h, c)];
      float2 w = tw[q * s1];
      w.y = -w.y;
      float2 y = cmul(x1, w);
      x1 = make_float2(x0.x - y.x, x0.y - y.y);
      x0 = make_float2(x0.x + y.x, x0.y + y.y);
      y = cmul(x3, w);
      x3 = make_float2(x2.x - y.x, x2.y - y.y);
      x2 = make_float2(x2.x + y.x, x2.y + y.y);
      float2 wa = tw[q * s2], wb = tw[(q + h) * s2];
      wa.y = -wa.y;
      wb.y = -wb.y;
      y = cmul(x2, wa);
      a[slot<KC>(i0, c)] = make_float2(x0.x + y.x, x0.y + y.y);
      a[slot<KC>(i0 + 2 * h, c)] = make_float2(x0.x - y.x, x0.y - y.y);
      y = cmul(x3, wb);
      a[slot<KC>(i0 + h, c)] = make_float2(x1.x + y.x, x1.y + y.y);
      a[slot<KC>(i0 + 3 * h, c)] = make_float2(x1.x - y.x, x1.y - y.y);
    }
    __syncthreads();
  }
  if (2 * h == P) {  // h = P/2 left over
    for (int id = threadIdx.x; id < h * KC; id += blockDim.x) {
      const int c = id % KC, j = id / KC;
      float2 w = tw[j];
      w.y = -w.y;
      const float2 u = a[slot<KC>(j, c)], v = cmul(a[slot<KC>(j + h, c)], w);
      a[slot<KC>(j, c)] = make_float2(u.x + v.x, u.y + v.y);
      a[slot<KC>(j + h, c)] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
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

// y = F x for n_lines A-lines of nt samples (x and y may alias).  Block b
// holds real lines 2 KC b .. 2 KC b + 2 KC - 1; complex line c carries real
// lines 2c (real part) and 2c + 1 (imaginary part).  hb: the filter's
// spectrum over NF, in bit-reversed order (NF floats).
template <int KC>
__global__ void __launch_bounds__(kFirThreads) k_fir_lines(const float *x, float *y, long long n_lines, int nt,
                                                           int NF, int lgNF, const float *__restrict__ hb) {
  extern __shared__ float2 sm[];
  float2 *tw = sm, *a = sm + (NF >> 1);
  const long long line0 = (long long)blockIdx.x * (2 * KC);
  load_twiddles(tw, NF);
  for (int i = threadIdx.x; i < KC * NF; i += blockDim.x) {
    const int c = i % KC, n = i / KC;
    const long long l0 = line0 + 2 * c, l1 = l0 + 1;
    float re = 0.0f, im = 0.0f;
    if (n < nt) {
      if (l0 < n_lines) re = x[l0 * nt + n];
      if (l1 < n_lines) im = x[l1 * nt + n];
    }
    a[slot<KC>(n, c)] = make_float2(re, im);
  }
  __syncthreads();
  dif_outer<KC>(a, tw, NF, lgNF);
  const int groups = NF >> 3;
  for (int id = threadIdx.x; id < groups * KC; id += blockDim.x)
    mid_group<KC>(a, id % groups, id / groups, reinterpret_cast<const float4 *>(hb));
  __syncthreads();
  dit_outer<KC>(a, tw, NF, lgNF);
  for (int i = threadIdx.x; i < KC * nt; i += blockDim.x) {
    const int c = i % KC, n = i / KC;
    const long long l0 = line0 + 2 * c, l1 = l0 + 1;
    const float2 v = a[slot<KC>(n, c)];
    if (l0 < n_lines) y[l0 * nt + n] = v.x;
    if (l1 < n_lines) y[l1 * nt + n] = v.y;
  }
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
  int NF = 8, lg = 3;  // at least one 8-point group
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
