// Lateral-FFT form of the forward and adjoint operators (FP32).
//
// A and A^T are 2-D correlations of the single-position slab with the volume
// over the scan grid (Methods, Efficient reconstruction based on scanning
// symmetries: the model is the same for every scanning position).  With the
// volume and the signals zero-padded to P x P, P a power of two with
// P >= max(py, px) + R, no circular wrap reaches the output window, and the
// correlation theorem restates both operators exactly per lateral frequency
// (v, u):
//   A:    s^(v,u,n) = sum_k S^(v,u,k,n) H^(v,u,k)
//   A^T:  H^(v,u,k) = sum_n S^(v,u,k,n) s^(v,u,n)
// The slab is mirror-symmetric in both lateral offsets (the patch set is;
// Results, axial symmetry), so its lateral DFT
//   S^(v,u,k,n) = sum_{b,a} S[b][a][k][n] cos(2 pi v b / P) cos(2 pi u a / P)
// is real and even in v and in u (and symmetric in (v, u) when dx = dy), and
// conj(S^) = S^.  Ŝ is therefore stored once per frequency orbit
// {(+-v, +-u)} (and (u, v)), each orbit row holding, for every depth k, the
// union band of samples [klo_k, klo_k + klen_k) over all lateral offsets.
//
// One application is five launches: FFT along x of real rows (half spectrum
// u in [0, P/2]), FFT along y, the per-orbit banded real matrix times up to
// four complex frequency vectors, inverse FFT along y, inverse FFT along x
// back to real rows (Hermitian extension) with zero fill outside the band.
// FFTs are radix-2 in shared memory with twiddles from sincospi; every sum
// runs in a fixed order, so results are deterministic.
#include <algorithm>
#include <set>
#include <vector>

#include "fft_dev.cuh"
#include "internal.cuh"

using namespace oam;

namespace oam {

struct FftLayout {
  int P = 0, lgP = 0, Q = 0;  // transform size, its log2, half-spectrum columns P/2 + 1
  int KC = 0;                 // channels per FFT block
  bool d4 = false;            // S^(v,u) = S^(u,v)
  int n_rep = 0;              // frequency orbits
  int NS = 0;                 // support length n_hi - n_lo
  int C = 0;                  // max(nz, NS): channels of the work buffers
  long long row_len = 0;      // sum_k klen_k: entries of one orbit row of S^
  long long row_stride = 0;   // row_len rounded up to 4 floats: each row starts on a 16-byte boundary
  int *d_klo = nullptr, *d_klen = nullptr;  // [nz] union band per depth (absolute samples)
  long long *d_koff = nullptr;              // [nz] offset of depth k in an orbit row
  int4 *d_members = nullptr;                // [n_rep] half-spectrum indices u*P + v (-1 unused)
  int2 *d_krange = nullptr;                 // [NS] depths [x, y) whose band can hold sample n_lo + j
  long long *d_noff = nullptr;              // [NS] offset of sample n_lo + j in a transposed orbit row
  long long row_len_t = 0;                  // sum_j (krange_j.y - krange_j.x)
  long long row_stride_t = 0;               // row_len_t rounded up to 4 floats
  float *d_shat_t = nullptr;                // [n_rep][row_stride_t]: S^ by sample, depths krange_j (adjoint)
  float *d_shat = nullptr;                  // [n_rep][row_stride]
  float2 *d_w1 = nullptr, *d_w2 = nullptr;  // [Q][P][C] work buffers
  double flops = 0;                         // flops of one application (matrix part + FFTs)
  double bytes = 0;                         // device bytes read + written per application
};

}  // namespace oam

namespace {

using namespace oam::fftdev;

constexpr int kFftThreads = 256;
constexpr int kApplyMaxThreads = 1024;
constexpr int kUnroll = 8;  // spectral products: independent row loads per lane in flight
constexpr int kFwdPhases = 2;  // forward products: lane groups of a warp that walk interleaved depths
constexpr int kFwdChunk = 256;  // forward products: samples per block (0: all samples of the orbit)
constexpr int kAdjChunk = 160;  // adjoint products: depths per block (0: all depths of the orbit)
constexpr int kBuildThreads = 128;


// Real rows -> half spectrum along x.  X[py][px][Ctot] (channels c0 .. c0+C-1
// used), Y[Q][py][C] complex.  Block (y, channel block of KC).  Channels l and
// l + KC/2 ride as the real and imaginary parts of one complex line; with
// Z = FFT(x + i y), X(u) = (Z(u) + conj Z(-u)) / 2 and Y(u) = (Z(u) - conj Z(-u)) / 2i.
template <int KC>
__global__ void __launch_bounds__(kFftThreads) k_fft_rows_r2c(const float *__restrict__ X, int py, int px, int Ctot,
                                                              int c0, int C, int P, int lgP, int Q,
                                                              float2 *__restrict__ Y) {
  constexpr int KH = KC / 2;  // complex lines
  extern __shared__ float2 sm[];
  float2 *tw = sm, *a = sm + (P >> 1);
  const int y = blockIdx.x, cb = blockIdx.y * KC;
  load_twiddles(tw, P);
  for (int i = threadIdx.x; i < P * KH; i += blockDim.x) {
    const int x = i / KH, l = i % KH;
    float re = 0.0f, im = 0.0f;
    if (x < px) {
      const float *row = X + ((size_t)y * px + x) * Ctot + c0 + cb;
      if (cb + l < C) re = row[l];
      if (cb + l + KH < C) im = row[l + KH];
    }
    a[bitrev(x, lgP) * KH + l] = make_float2(re, im);
  }
  fft_lines<KH>(a, tw, P, lgP, false);
  for (int i = threadIdx.x; i < Q * KC; i += blockDim.x) {
    const int u = i / KC, c = i % KC, l = c % KH;
    if (cb + c >= C) continue;
    const float2 z = a[u * KH + l], w = a[((P - u) & (P - 1)) * KH + l];
    Y[((size_t)u * py + y) * C + cb + c] = c < KH ? make_float2(0.5f * (z.x + w.x), 0.5f * (z.y - w.y))
                                                  : make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
  }
}

// Complex transform along the row index of Z[Q][nin][C] -> W[Q][nout][C]
// (rows >= nin read as zero, rows >= nout dropped).  Block (u, channel block).
template <int KC>
__global__ void __launch_bounds__(kFftThreads) k_fft_cols(const float2 *__restrict__ Z, int nin, int nout, int C, int P,
                                                          int lgP, int inverse, float2 *__restrict__ W) {
  extern __shared__ float2 sm[];
  float2 *tw = sm, *a = sm + (P >> 1);
  const int u = blockIdx.x, cb = blockIdx.y * KC;
  load_twiddles(tw, P);
  for (int i = threadIdx.x; i < P * KC; i += blockDim.x) {
    const int r = i / KC, c = i % KC;
    float2 v = make_float2(0.0f, 0.0f);
    if (r < nin && cb + c < C) v = Z[((size_t)u * nin + r) * C + cb + c];
    a[bitrev(r, lgP) * KC + c] = v;
  }
  fft_lines<KC>(a, tw, P, lgP, inverse != 0);
  for (int i = threadIdx.x; i < nout * KC; i += blockDim.x) {
    const int r = i / KC, c = i % KC;
    if (cb + c < C) W[((size_t)u * nout + r) * C + cb + c] = a[r * KC + c];
  }
}

// Half spectrum along x -> real rows, scaled by 1/P^2.  Z[Q][py][C] holds
// channels c0 .. c0+C-1 of the output X[py][px][Ctot]; every other output
// channel is written as zero.  Block (y, output channel block of KC).
// Channels l and l + KC/2 share one complex line W = X + i Y (each extended
// Hermitian, the imaginary parts of its u = 0 and u = P/2 terms dropped): the
// inverse transform's real and imaginary parts are the two real rows.
template <int KC>
__global__ void __launch_bounds__(kFftThreads) k_fft_rows_c2r(const float2 *__restrict__ Z, int py, int px, int Ctot,
                                                              int c0, int C, int P, int lgP, int Q,
                                                              float scale, float *__restrict__ X) {
  constexpr int KH = KC / 2;
  extern __shared__ float2 sm[];
  float2 *tw = sm, *a = sm + (P >> 1);
  const int y = blockIdx.x, ob = blockIdx.y * KC;
  if (ob >= c0 + C || ob + KC <= c0) {  // block entirely outside the band: zeros
    for (int i = threadIdx.x; i < px * KC; i += blockDim.x) {
      const int x = i / KC, c = i % KC;
      if (ob + c < Ctot) X[((size_t)y * px + x) * Ctot + ob + c] = 0.0f;
    }
    return;
  }
  load_twiddles(tw, P);
  for (int i = threadIdx.x; i < P * KH; i += blockDim.x) {
    const int f = i / KH, l = i % KH;
    const int fh = f < Q ? f : P - f;  // Hermitian source column
    float2 xs = make_float2(0.0f, 0.0f), ys = make_float2(0.0f, 0.0f);
    const int zx = ob + l - c0, zy = ob + l + KH - c0;
    if (zx >= 0 && zx < C) xs = Z[((size_t)fh * py + y) * C + zx];
    if (zy >= 0 && zy < C) ys = Z[((size_t)fh * py + y) * C + zy];
    if (f == 0 || f == (P >> 1)) {
      xs.y = 0.0f;
      ys.y = 0.0f;
    } else if (f >= Q) {
      xs.y = -xs.y;
      ys.y = -ys.y;
    }
    a[bitrev(f, lgP) * KH + l] = make_float2(xs.x - ys.y, xs.y + ys.x);
  }
  fft_lines<KH>(a, tw, P, lgP, true);
  for (int i = threadIdx.x; i < px * KC; i += blockDim.x) {
    const int x = i / KC, c = i % KC, l = c % KH;
    const int oc = ob + c, zc = oc - c0;
    if (oc >= Ctot) continue;
    const float2 v = a[x * KH + l];
    X[((size_t)y * px + x) * Ctot + oc] = (zc >= 0 && zc < C) ? (c < KH ? v.x : v.y) * scale : 0.0f;
  }
}

// ---- transforms in register passes (P >= 16) ------------------------------
// The kernels above move every point through shared memory once per two
// radix-2 stages and scatter it to its bit-reversed slot first.  The kernels
// below run up to four stages per pass in registers: a forward transform is
// decimation in frequency (natural order in, bit-reversed out: the point at
// position i ends as frequency bitrev(i), which goes to global row bitrev(i)),
// an inverse transform decimation in time (position i loads frequency
// bitrev(i), natural order out), so no permutation pass is needed, the first
// pass reads global memory and the last writes it.  Passes cover stages
// k .. k + r - 1 (spans 2^k .. 2^(k+r-1)) with k a multiple of 4: the first
// forward pass has r0 = log2 P - 4 (ceil(log2 P / 4) - 1) stages, every other
// pass four.

// Shared-memory slot of point i of line l among KL lines: lines fastest, and
// for KL < 16 a pad of KL slots after every 16 points, so that the 16 lines x
// points a half-warp touches in a pass fall in distinct banks.
template <int KL>
__device__ __forceinline__ int xslot(int i, int l) {
  return i * KL + l + (KL < 16 ? (i >> 4) * KL : 0);
}
template <int KL>
__host__ __device__ constexpr size_t xslots(int P) {
  return (size_t)P * KL + (KL < 16 ? (size_t)(P >> 4) * KL : 0);
}

// One pass of r stages over the points i0 + m 2^k (m < 2^r) of each group
// (line l, q < 2^k, block blk; i0 = blk 2^(k+r) + q).  Forward (decimation in
// frequency, spans from large to small): span S = 2^(k+j) maps (u, w) at
// (n, n + S) to (u + w, (u - w) W_2S^(n mod S)), n mod S = q + (m mod 2^j) 2^k,
// twiddle W_2S^q W_2^(j+1)^(m mod 2^j), the first factor a power of
// b = W_2^(k+r)^q (one sincospif, then squarings).  Inverse (decimation in
// time, spans from small to large, sign +1): (u, w) go to (u + w conj(W),
// u - w conj(W)).  src(i, l) yields point i before the pass, dst(i, l, v)
// takes it after.
template <int KL, int r, bool kForward, class Src, class Dst>
__device__ __forceinline__ void xpass(int P, int k, Src src, Dst dst) {
  constexpr int R = 1 << r;
  const int groups = P >> r;
  for (int id = threadIdx.x; id < groups * KL; id += blockDim.x) {
    const int l = id % KL, t = id / KL;
    const int q = t & ((1 << k) - 1), blk = t >> k;
    const int i0 = (blk << (k + r)) | q;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = src(i0 + (m << k), l);
    float2 pw[r];
    sincospif(-2.0f * (float)q / (float)(1 << (k + r)), &pw[r - 1].y, &pw[r - 1].x);
#pragma unroll
    for (int j = r - 2; j >= 0; --j) pw[j] = cmul(pw[j + 1], pw[j + 1]);
    if (kForward) {
#pragma unroll
      for (int j = r - 1; j >= 0; --j) {
        const int S = 1 << j;
#pragma unroll
        for (int m = 0; m < R; ++m) {
          if (m & S) continue;
          const float2 u = v[m], w = v[m + S];
          v[m] = make_float2(u.x + w.x, u.y + w.y);
          const int um = m & (S - 1);
          const float2 tw = um == 0 ? pw[j] : cmul(pw[j], w16(2 * S, um));
          v[m + S] = cmul(make_float2(u.x - w.x, u.y - w.y), tw);
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < r; ++j) {
        const int S = 1 << j;
#pragma unroll
        for (int m = 0; m < R; ++m) {
          if (m & S) continue;
          const int um = m & (S - 1);
          const float2 tw = um == 0 ? pw[j] : cmul(pw[j], w16(2 * S, um));
          const float2 u = v[m], w = cmul(v[m + S], make_float2(tw.x, -tw.y));
          v[m] = make_float2(u.x + w.x, u.y + w.y);
          v[m + S] = make_float2(u.x - w.x, u.y - w.y);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) dst(i0 + (m << k), l, v[m]);
  }
}

// A whole transform of KL lines of P = 2^lgP points (lgP >= 4) through the
// shared slots `a`: `first` reads the input (forward: natural point i;
// inverse: the point at position i, i.e. frequency bitrev(i)), `last` takes
// position i's result (forward: frequency bitrev(i); inverse: point i).  With
// kLastToSmem the last pass writes the slots too (followed by a barrier) and
// `last` is not called.
template <int KL, bool kForward, bool kLastToSmem, class First, class Last>
__device__ __forceinline__ void xtransform(float2 *a, int P, int lgP, First first, Last last) {
  const int np = (lgP + 3) / 4, r0 = lgP - 4 * (np - 1);
  auto from_smem = [&](int i, int l) { return a[xslot<KL>(i, l)]; };
  auto to_smem = [&](int i, int l, float2 v) { a[xslot<KL>(i, l)] = v; };
  // pass p covers stages [kf, kf + rr): forward passes run p = 0 .. np-1 with
  // kf = 4 (np-1-p) (the first has r0 stages), inverse passes the reverse
  for (int pi = 0; pi < np; ++pi) {
    const int pp = kForward ? pi : np - 1 - pi;  // which stage block
    const int kf = 4 * (np - 1 - pp), rr = pp == 0 ? r0 : 4;
    const bool is_first = pi == 0, is_last = pi == np - 1;
    if (is_first && is_last) {
      if (kLastToSmem) {
        switch (rr) {
          case 1: xpass<KL, 1, kForward>(P, kf, first, to_smem); break;
          case 2: xpass<KL, 2, kForward>(P, kf, first, to_smem); break;
          case 3: xpass<KL, 3, kForward>(P, kf, first, to_smem); break;
          default: xpass<KL, 4, kForward>(P, kf, first, to_smem); break;
        }
      } else {
        switch (rr) {
          case 1: xpass<KL, 1, kForward>(P, kf, first, last); break;
          case 2: xpass<KL, 2, kForward>(P, kf, first, last); break;
          case 3: xpass<KL, 3, kForward>(P, kf, first, last); break;
          default: xpass<KL, 4, kForward>(P, kf, first, last); break;
        }
      }
    } else if (is_first) {
      switch (rr) {
        case 1: xpass<KL, 1, kForward>(P, kf, first, to_smem); break;
        case 2: xpass<KL, 2, kForward>(P, kf, first, to_smem); break;
        case 3: xpass<KL, 3, kForward>(P, kf, first, to_smem); break;
        default: xpass<KL, 4, kForward>(P, kf, first, to_smem); break;
      }
    } else if (is_last && !kLastToSmem) {
      switch (rr) {
        case 1: xpass<KL, 1, kForward>(P, kf, from_smem, last); break;
        case 2: xpass<KL, 2, kForward>(P, kf, from_smem, last); break;
        case 3: xpass<KL, 3, kForward>(P, kf, from_smem, last); break;
        default: xpass<KL, 4, kForward>(P, kf, from_smem, last); break;
      }
    } else {
      switch (rr) {
        case 1: xpass<KL, 1, kForward>(P, kf, from_smem, to_smem); break;
        case 2: xpass<KL, 2, kForward>(P, kf, from_smem, to_smem); break;
        case 3: xpass<KL, 3, kForward>(P, kf, from_smem, to_smem); break;
        default: xpass<KL, 4, kForward>(P, kf, from_smem, to_smem); break;
      }
    }
    if (!is_last || kLastToSmem) __syncthreads();
  }
}

// k_fft_rows_r2c in register passes (P >= 16): same arguments and results.
template <int KC>
__global__ void __launch_bounds__(kFftThreads) k_xfft_rows_r2c(const float *__restrict__ X, int py, int px, int Ctot,
                                                               int c0, int C, int P, int lgP, int Q,
                                                               float2 *__restrict__ Y) {
  constexpr int KH = KC / 2;
  extern __shared__ float2 sm[];
  float2 *a = sm;
  const int y = blockIdx.x, cb = blockIdx.y * KC;
  const float *row = X + (size_t)y * px * Ctot + c0 + cb;
  auto load = [&](int x, int l) {
    float re = 0.0f, im = 0.0f;
    if (x < px) {
      const float *p = row + (size_t)x * Ctot;
      if (cb + l < C) re = p[l];
      if (cb + l + KH < C) im = p[l + KH];
    }
    return make_float2(re, im);
  };
  auto none = [](int, int, float2) {};
  xtransform<KH, true, true>(a, P, lgP, load, none);
  for (int i = threadIdx.x; i < Q * KC; i += blockDim.x) {
    const int u = i / KC, c = i % KC, l = c % KH;
    if (cb + c >= C) continue;
    const float2 z = a[xslot<KH>(bitrev(u, lgP), l)], w = a[xslot<KH>(bitrev((P - u) & (P - 1), lgP), l)];
    Y[((size_t)u * py + y) * C + cb + c] = c < KH ? make_float2(0.5f * (z.x + w.x), 0.5f * (z.y - w.y))
                                                  : make_float2(0.5f * (z.y + w.y), 0.5f * (w.x - z.x));
  }
}

// k_fft_cols in register passes (P >= 16): same arguments and results.
template <int KC, bool kInverse>
__global__ void __launch_bounds__(kFftThreads) k_xfft_cols(const float2 *__restrict__ Z, int nin, int nout, int C,
                                                           int P, int lgP, float2 *__restrict__ W) {
  extern __shared__ float2 sm[];
  const int u = blockIdx.x, cb = blockIdx.y * KC;
  const float2 *zin = Z + (size_t)u * nin * C + cb;
  float2 *wout = W + (size_t)u * nout * C + cb;
  auto load = [&](int i, int l) {
    const int row = kInverse ? bitrev(i, lgP) : i;
    return (row < nin && cb + l < C) ? zin[(size_t)row * C + l] : make_float2(0.0f, 0.0f);
  };
  auto store = [&](int i, int l, float2 v) {
    const int row = kInverse ? i : bitrev(i, lgP);
    if (row < nout && cb + l < C) wout[(size_t)row * C + l] = v;
  };
  xtransform<KC, !kInverse, false>(sm, P, lgP, load, store);
}

// k_fft_rows_c2r in register passes (P >= 16): same arguments and results.
template <int KC>
__global__ void __launch_bounds__(kFftThreads) k_xfft_rows_c2r(const float2 *__restrict__ Z, int py, int px, int Ctot,
                                                               int c0, int C, int P, int lgP, int Q, float scale,
                                                               float *__restrict__ X) {
  constexpr int KH = KC / 2;
  extern __shared__ float2 sm[];
  const int y = blockIdx.x, ob = blockIdx.y * KC;
  if (ob >= c0 + C || ob + KC <= c0) {  // block entirely outside the band: zeros
    for (int i = threadIdx.x; i < px * KC; i += blockDim.x) {
      const int x = i / KC, c = i % KC;
      if (ob + c < Ctot) X[((size_t)y * px + x) * Ctot + ob + c] = 0.0f;
    }
    return;
  }
  // position i takes frequency f = bitrev(i) of W = X + i Y, the two real
  // channels' Hermitian-extended spectra (imaginary parts of f = 0, P/2 dropped)
  auto load = [&](int i, int l) {
    const int f = bitrev(i, lgP);
    const int fh = f < Q ? f : P - f;
    float2 xs = make_float2(0.0f, 0.0f), ys = make_float2(0.0f, 0.0f);
    const int zx = ob + l - c0, zy = ob + l + KH - c0;
    if (zx >= 0 && zx < C) xs = Z[((size_t)fh * py + y) * C + zx];
    if (zy >= 0 && zy < C) ys = Z[((size_t)fh * py + y) * C + zy];
    if (f == 0 || f == (P >> 1)) {
      xs.y = 0.0f;
      ys.y = 0.0f;
    } else if (f >= Q) {
      xs.y = -xs.y;
      ys.y = -ys.y;
    }
    return make_float2(xs.x - ys.y, xs.y + ys.x);
  };
  auto store = [&](int x, int l, float2 v) {
    if (x >= px) return;
    float *p = X + ((size_t)y * px + x) * Ctot;
    const int o0 = ob + l, o1 = ob + l + KH;
    if (o0 < Ctot) p[o0] = (o0 - c0 >= 0 && o0 - c0 < C) ? v.x * scale : 0.0f;
    if (o1 < Ctot) p[o1] = (o1 - c0 >= 0 && o1 - c0 < C) ? v.y * scale : 0.0f;
  };
  xtransform<KH, false, false>(sm, P, lgP, load, store);
}

// Forward, per frequency orbit r: s^_f[j] = sum_k S^_r[k][n - klo_k] H^_f[k]
// for the orbit's member frequencies f, n = n_lo + j; thread j visits the
// depths [kr_j.x, kr_j.y) whose band holds n.  Block per orbit.
__global__ void __launch_bounds__(kApplyMaxThreads) k_fft_apply_fwd(const float *__restrict__ shat, long long row_len,
                                                        const int4 *__restrict__ members,
                                                        const int *__restrict__ klo, const int *__restrict__ klen,
                                                        const long long *__restrict__ koff,
                                                        const int2 *__restrict__ krange, int nz, int n_lo, int NS,
                                                        const float2 *__restrict__ Hh, float2 *__restrict__ sh) {
  extern __shared__ float4 smf[];
  float4 *Hs = smf;                                  // [nz][2]: members (0, 1) and (2, 3), (re, im) pairs
  int *s_lo = reinterpret_cast<int *>(Hs + 2 * nz);   // [nz]
  int *s_len = s_lo + nz;                             // [nz]
  long long *s_off = reinterpret_cast<long long *>(s_len + nz);  // [nz]: 40 nz bytes in, 8-byte aligned
  // linear grid, chunk fastest: an orbit's sample chunks run back to back and share its vectors in L2
  const int nch = kFwdChunk > 0 ? (NS + kFwdChunk - 1) / kFwdChunk : 1;
  const int r = (int)(blockIdx.x / nch), chunk = (int)(blockIdx.x % nch);
  const int4 mem = members[r];
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    const float2 z = make_float2(0.0f, 0.0f);
    const float2 h0 = mem.x >= 0 ? Hh[(size_t)mem.x * nz + k] : z, h1 = mem.y >= 0 ? Hh[(size_t)mem.y * nz + k] : z;
    const float2 h2 = mem.z >= 0 ? Hh[(size_t)mem.z * nz + k] : z, h3 = mem.w >= 0 ? Hh[(size_t)mem.w * nz + k] : z;
    Hs[2 * k] = make_float4(h0.x, h0.y, h1.x, h1.y);
    Hs[2 * k + 1] = make_float4(h2.x, h2.y, h3.x, h3.y);
    s_lo[k] = klo[k];
    s_len[k] = klen[k];
    s_off[k] = koff[k];
  }
  __syncthreads();
  const float *row = shat + (size_t)r * row_len;
  constexpr int kLanes = 32 / kFwdPhases;  // samples per warp
  const int lane = threadIdx.x & 31, sub = lane % kLanes, ph = lane / kLanes;
  const int jb = kFwdChunk > 0 ? chunk * kFwdChunk : 0;
  const int je = kFwdChunk > 0 ? min(NS, jb + kFwdChunk) : NS;
  // a warp serves kLanes samples; its lane groups walk interleaved depths of
  // the warp's common depth range (coalesced row reads), then add their sums
  for (int g0 = jb + (threadIdx.x >> 5) * kLanes; g0 < je; g0 += (blockDim.x >> 5) * kLanes) {
    const int j = g0 + sub;
    const bool live = j < je;
    const int n = n_lo + j;
    const int2 kr = live ? krange[j] : make_int2(nz, 0);
    const int k0 = __reduce_min_sync(0xffffffffu, kr.x), k1 = __reduce_max_sync(0xffffffffu, kr.y);
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
    int k = k0 + ph;
    for (; k + kFwdPhases * (kUnroll - 1) < k1; k += kFwdPhases * kUnroll) {  // kUnroll loads in flight per lane
      float sv[kUnroll];
#pragma unroll
      for (int q = 0; q < kUnroll; ++q) {
        const int kk = k + kFwdPhases * q, d = n - s_lo[kk];
        sv[q] = (live && (unsigned)d < (unsigned)s_len[kk]) ? __ldg(row + s_off[kk] + d) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < kUnroll; ++q) {
        const float4 a = Hs[2 * (k + kFwdPhases * q)], b = Hs[2 * (k + kFwdPhases * q) + 1];
        acc[0] = fmaf(sv[q], a.x, acc[0]);
        acc[1] = fmaf(sv[q], a.y, acc[1]);
        acc[2] = fmaf(sv[q], a.z, acc[2]);
        acc[3] = fmaf(sv[q], a.w, acc[3]);
        acc[4] = fmaf(sv[q], b.x, acc[4]);
        acc[5] = fmaf(sv[q], b.y, acc[5]);
        acc[6] = fmaf(sv[q], b.z, acc[6]);
        acc[7] = fmaf(sv[q], b.w, acc[7]);
      }
    }
    for (; k < k1; k += kFwdPhases) {
      const int d = n - s_lo[k];
      const float sv = (live && (unsigned)d < (unsigned)s_len[k]) ? __ldg(row + s_off[k] + d) : 0.0f;
      const float4 a = Hs[2 * k], b = Hs[2 * k + 1];
      acc[0] = fmaf(sv, a.x, acc[0]);
      acc[1] = fmaf(sv, a.y, acc[1]);
      acc[2] = fmaf(sv, a.z, acc[2]);
      acc[3] = fmaf(sv, a.w, acc[3]);
      acc[4] = fmaf(sv, b.x, acc[4]);
      acc[5] = fmaf(sv, b.y, acc[5]);
      acc[6] = fmaf(sv, b.z, acc[6]);
      acc[7] = fmaf(sv, b.w, acc[7]);
    }
#pragma unroll
    for (int off = 16; off >= kLanes; off >>= 1)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    if (!live || ph != 0) continue;
    if (mem.x >= 0) sh[(size_t)mem.x * NS + j] = make_float2(acc[0], acc[1]);
    if (mem.y >= 0) sh[(size_t)mem.y * NS + j] = make_float2(acc[2], acc[3]);
    if (mem.z >= 0) sh[(size_t)mem.z * NS + j] = make_float2(acc[4], acc[5]);
    if (mem.w >= 0) sh[(size_t)mem.w * NS + j] = make_float2(acc[6], acc[7]);
  }
}

// Adjoint, per frequency orbit r: H^_f[k] = sum_n S^_r[k][n] s^_f[n - n_lo], from
// the orbit's row by sample (entries of sample n_lo + j are depths krange_j).
// Thread k; every lane of a warp walks the same samples (coalesced reads).
__global__ void __launch_bounds__(kApplyMaxThreads) k_fft_apply_adj(const float *__restrict__ shat_t,
                                                                    long long row_len_t,
                                                                    const int4 *__restrict__ members,
                                                                    const int *__restrict__ klo,
                                                                    const int *__restrict__ klen,
                                                                    const int2 *__restrict__ krange,
                                                                    const long long *__restrict__ noff, int nz,
                                                                    int n_lo, int NS, const float2 *__restrict__ sh,
                                                                    float2 *__restrict__ Hh) {
  extern __shared__ float4 sma[];
  float4 *Ss = sma;                                      // [NS][2]: members (0, 1) and (2, 3)
  int2 *s_kr = reinterpret_cast<int2 *>(Ss + 2 * NS);     // [NS]
  long long *s_no = reinterpret_cast<long long *>(s_kr + NS);  // [NS]
  // linear grid, chunk fastest: an orbit's depth chunks run back to back
  const int nch = kAdjChunk > 0 ? (nz + kAdjChunk - 1) / kAdjChunk : 1;
  const int r = (int)(blockIdx.x / nch), chunk = (int)(blockIdx.x % nch);
  const int kb = kAdjChunk > 0 ? chunk * kAdjChunk : 0, ke = kAdjChunk > 0 ? min(nz, kb + kAdjChunk) : nz;
  const int4 mem = members[r];
  for (int j = threadIdx.x; j < NS; j += blockDim.x) {
    const float2 z = make_float2(0.0f, 0.0f);
    const float2 x0 = mem.x >= 0 ? sh[(size_t)mem.x * NS + j] : z, x1 = mem.y >= 0 ? sh[(size_t)mem.y * NS + j] : z;
    const float2 x2 = mem.z >= 0 ? sh[(size_t)mem.z * NS + j] : z, x3 = mem.w >= 0 ? sh[(size_t)mem.w * NS + j] : z;
    Ss[2 * j] = make_float4(x0.x, x0.y, x1.x, x1.y);
    Ss[2 * j + 1] = make_float4(x2.x, x2.y, x3.x, x3.y);
    s_kr[j] = krange[j];
    s_no[j] = noff[j];
  }
  __syncthreads();
  const float *row = shat_t + (size_t)r * row_len_t;
  const int lane = threadIdx.x & 31, sub = lane & 15, ph = lane >> 4;
  // a warp serves 16 depths; its two half-warps walk alternate samples of the
  // warp's common sample range (coalesced reads), then add their sums
  for (int g0 = kb + (threadIdx.x >> 5) * 16; g0 < ke; g0 += (blockDim.x >> 5) * 16) {
    const int k = g0 + sub;
    const bool live = k < ke && klen[k] > 0;
    const int lo = live ? klo[k] - n_lo : NS, hi = live ? klo[k] - n_lo + klen[k] : 0;
    const int j0 = __reduce_min_sync(0xffffffffu, lo), j1 = __reduce_max_sync(0xffffffffu, hi);
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
    int j = j0 + ph;
    for (; j + 2 * (kUnroll - 1) < j1; j += 2 * kUnroll) {  // kUnroll loads in flight per lane
      float sv[kUnroll];
#pragma unroll
      for (int q = 0; q < kUnroll; ++q) {
        const int jj = j + 2 * q;
        const int2 kr = s_kr[jj];
        sv[q] = (k >= kr.x && k < kr.y) ? __ldg(row + s_no[jj] + (k - kr.x)) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < kUnroll; ++q) {
        const float4 a = Ss[2 * (j + 2 * q)], b = Ss[2 * (j + 2 * q) + 1];
        acc[0] = fmaf(sv[q], a.x, acc[0]);
        acc[1] = fmaf(sv[q], a.y, acc[1]);
        acc[2] = fmaf(sv[q], a.z, acc[2]);
        acc[3] = fmaf(sv[q], a.w, acc[3]);
        acc[4] = fmaf(sv[q], b.x, acc[4]);
        acc[5] = fmaf(sv[q], b.y, acc[5]);
        acc[6] = fmaf(sv[q], b.z, acc[6]);
        acc[7] = fmaf(sv[q], b.w, acc[7]);
      }
    }
    for (; j < j1; j += 2) {
      const int2 kr = s_kr[j];
      const float sv = (k >= kr.x && k < kr.y) ? __ldg(row + s_no[j] + (k - kr.x)) : 0.0f;
      const float4 a = Ss[2 * j], b = Ss[2 * j + 1];
      acc[0] = fmaf(sv, a.x, acc[0]);
      acc[1] = fmaf(sv, a.y, acc[1]);
      acc[2] = fmaf(sv, a.z, acc[2]);
      acc[3] = fmaf(sv, a.w, acc[3]);
      acc[4] = fmaf(sv, b.x, acc[4]);
      acc[5] = fmaf(sv, b.y, acc[5]);
      acc[6] = fmaf(sv, b.z, acc[6]);
      acc[7] = fmaf(sv, b.w, acc[7]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 16);
    if (k >= ke || ph != 0) continue;
    if (mem.x >= 0) Hh[(size_t)mem.x * nz + k] = make_float2(acc[0], acc[1]);
    if (mem.y >= 0) Hh[(size_t)mem.y * nz + k] = make_float2(acc[2], acc[3]);
    if (mem.z >= 0) Hh[(size_t)mem.z * nz + k] = make_float2(acc[4], acc[5]);
    if (mem.w >= 0) Hh[(size_t)mem.w * nz + k] = make_float2(acc[6], acc[7]);
  }
}

// ---------------------------------------------------------------- S^ build
// Pass 1: T[b'][u][e] = sum_{a'=0..R} w_a' cos(2 pi u a' / P) S[b'][a'][k_e][n_e]
// for every row entry e = (k_e, n_e); w_0 = 1, w_{>0} = 2 (the +-a' pair).
// Block (entry block, b').
__global__ void __launch_bounds__(kBuildThreads) k_shat_pass1(const float *__restrict__ band,
                                                              const int *__restrict__ band_lo,
                                                              const int *__restrict__ band_hi, int band_w,
                                                              const int *__restrict__ tap_orbit, int R, int W,
                                                              int nz, const int2 *__restrict__ entry_kn,
                                                              long long row_len, int P, int Q,
                                                              float *__restrict__ T) {
  extern __shared__ float smb[];
  float *cosT = smb;           // [P]
  float *sv = smb + P;         // [R+1][blockDim]: weighted slab values of this thread's entry
  for (int m = threadIdx.x; m < P; m += blockDim.x) cosT[m] = cospif(2.0f * (float)m / (float)P);
  __syncthreads();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int bp = blockIdx.y;
  if (e >= row_len) return;
  const int2 kn = entry_kn[e];
  const int ts = blockDim.x, tid = threadIdx.x;
  for (int ap = 0; ap <= R; ++ap) {
    const int o = tap_orbit[(bp + R) * W + (ap + R)];
    const int lo = band_lo[o * nz + kn.x], hi = band_hi[o * nz + kn.x];
    float v = 0.0f;
    if (kn.y >= lo && kn.y < hi) v = band[((size_t)o * nz + kn.x) * band_w + (kn.y - lo)];
    sv[ap * ts + tid] = ap == 0 ? v : 2.0f * v;
  }
  for (int u = 0; u < Q; ++u) {
    float acc = 0.0f;
    for (int ap = 0; ap <= R; ++ap) acc = fmaf(cosT[(u * ap) & (P - 1)], sv[ap * ts + tid], acc);
    T[((size_t)bp * Q + u) * row_len + e] = acc;
  }
}

// Pass 2: S^[r][e] = sum_{b'=0..R} w_b' cos(2 pi v0 b' / P) T[b'][u0][e] for
// every orbit r = (v0, u0) with this u0.  Block (entry block, u0).
__global__ void __launch_bounds__(kBuildThreads) k_shat_pass2(const float *__restrict__ T, long long row_len, int R,
                                                              int P, int Q, const int *__restrict__ rep_of,
                                                              const int2 *__restrict__ entry_kn, int n_lo,
                                                              const int2 *__restrict__ krange,
                                                              const long long *__restrict__ noff,
                                                              long long stride, long long stride_t,
                                                              float *__restrict__ shat, float *__restrict__ shat_t) {
  extern __shared__ float smb[];
  float *cosT = smb;    // [P]
  float *tv = smb + P;  // [R+1][blockDim]
  for (int m = threadIdx.x; m < P; m += blockDim.x) cosT[m] = cospif(2.0f * (float)m / (float)P);
  __syncthreads();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int u0 = blockIdx.y;
  if (e >= row_len) return;
  const int ts = blockDim.x, tid = threadIdx.x;
  for (int bp = 0; bp <= R; ++bp) {
    const float t = T[((size_t)bp * Q + u0) * row_len + e];
    tv[bp * ts + tid] = bp == 0 ? t : 2.0f * t;
  }
  const int2 kn = entry_kn[e];
  const int jn = kn.y - n_lo;
  const long long et = noff[jn] + (kn.x - krange[jn].x);  // same entry in the row by sample
  for (int v0 = 0; v0 < Q; ++v0) {
    const int r = rep_of[v0 * Q + u0];
    if (r < 0) continue;
    float acc = 0.0f;
    for (int bp = 0; bp <= R; ++bp) acc = fmaf(cosT[(v0 * bp) & (P - 1)], tv[bp * ts + tid], acc);
    shat[(size_t)r * stride + e] = acc;
    shat_t[(size_t)r * stride_t + et] = acc;
  }
}

size_t fft_smem(int P, int KC) { return sizeof(float2) * ((size_t)(P >> 1) + (size_t)P * KC); }

// Host tables of the lateral-FFT layout, planned from the model's bands.
struct FftPlan {
  std::vector<int> klo, klen;
  std::vector<long long> koff, noff;
  std::vector<int2> krange, entry_kn;
  std::vector<int> rep_of;
  std::vector<int4> members;
};

// Fill L's sizes and the host tables (no device call).
oam_status fft_plan(const oam_model *m, FftLayout *L, FftPlan &pl) {
  const int R = m->R, W = m->W, nz = m->grid.nz;
  const int need = std::max(m->grid.py, m->grid.px) + R;
  int P = 2, lgP = 1;
  while (P < need) {
    P <<= 1;
    ++lgP;
  }
  if (P > 2048) return OAM_ERR_UNSUPPORTED;
  L->P = P;
  L->lgP = lgP;
  L->Q = P / 2 + 1;
  L->KC = std::max(2, std::min(16, 4096 / P));
  const int Q = L->Q;
  // D4 when the tap -> orbit map is symmetric under b <-> a
  L->d4 = true;
  for (int b = -R; b <= R && L->d4; ++b)
    for (int a = -R; a <= R; ++a)
      if (m->h_tap_orbit[(b + R) * W + (a + R)] != m->h_tap_orbit[(a + R) * W + (b + R)]) {
        L->d4 = false;
        break;
      }
  // union band per depth over all orbits
  std::vector<int> &klo = pl.klo, &klen = pl.klen;
  std::vector<long long> &koff = pl.koff;
  klo.assign(nz, 0);
  klen.assign(nz, 0);
  koff.assign(nz, 0);
  long long row = 0;
  for (int k = 0; k < nz; ++k) {
    int lo = 1 << 30, hi = -1;
    for (int o = 0; o < m->n_orb; ++o) {
      const int bl = m->h_band_lo[(size_t)o * nz + k], bh = m->h_band_hi[(size_t)o * nz + k];
      if (bh > bl) {
        lo = std::min(lo, bl);
        hi = std::max(hi, bh);
      }
    }
    if (hi <= lo) lo = hi = m->n_lo;
    klo[k] = lo;
    klen[k] = hi - lo;
    koff[k] = row;
    row += hi - lo;
  }
  L->row_len = std::max<long long>(row, 1);
  L->row_stride = (L->row_len + 3) & ~3LL;
  L->NS = std::max(1, m->n_hi - m->n_lo);
  std::vector<int2> &krange = pl.krange;
  krange.assign(L->NS, make_int2(0, 0));
  for (int j = 0; j < L->NS; ++j) {
    const int n = m->n_lo + j;
    int kf = nz, kl = -1;
    for (int k = 0; k < nz; ++k)
      if (n >= klo[k] && n < klo[k] + klen[k]) {
        kf = std::min(kf, k);
        kl = std::max(kl, k);
      }
    krange[j] = kl >= kf ? make_int2(kf, kl + 1) : make_int2(0, 0);
  }
  std::vector<long long> &noff = pl.noff;
  noff.assign(L->NS, 0);
  long long rowt = 0;
  for (int j = 0; j < L->NS; ++j) {
    noff[j] = rowt;
    rowt += krange[j].y - krange[j].x;
  }
  L->row_len_t = std::max<long long>(rowt, 1);
  L->row_stride_t = (L->row_len_t + 3) & ~3LL;
  L->C = std::max(nz, L->NS);
  std::vector<int2> &entry_kn = pl.entry_kn;
  entry_kn.assign((size_t)L->row_len, make_int2(0, 0));
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < klen[k]; ++j) entry_kn[(size_t)koff[k] + j] = make_int2(k, klo[k] + j);
  // frequency orbits and their members in the half spectrum (index u*P + v)
  std::vector<int> &rep_of = pl.rep_of;
  std::vector<int4> &members = pl.members;
  rep_of.assign((size_t)Q * Q, -1);
  members.clear();
  long long covered = 0;
  for (int u0 = 0; u0 < Q; ++u0)
    for (int v0 = 0; v0 < (L->d4 ? u0 + 1 : Q); ++v0) {
      std::set<int> fs;
      for (int v : {v0, (P - v0) % P}) fs.insert(u0 * P + v);
      if (L->d4)
        for (int v : {u0, (P - u0) % P}) fs.insert(v0 * P + v);
      int4 mm = make_int4(-1, -1, -1, -1);
      int *slot = &mm.x;
      int i = 0;
      for (int f : fs) slot[i++] = f;
      covered += i;
      rep_of[(size_t)v0 * Q + u0] = (int)members.size();
      members.push_back(mm);
    }
  if (covered != (long long)Q * P) return OAM_ERR_DEVICE;  // orbit plan must cover the half spectrum once
  L->n_rep = (int)members.size();
  return OAM_OK;
}

// Device bytes fft_build allocates and keeps (host only).
oam_status fft_layout_bytes(const FftLayout &L, const FftPlan &pl, int nz, size_t *bytes) {
  *bytes = alloc_bytes<int>(nz) * 2 + alloc_bytes<long long>(nz) + alloc_bytes<int4>(pl.members.size()) +
           alloc_bytes<int2>(L.NS) + alloc_bytes<long long>(L.NS) +
           alloc_bytes<float>((size_t)L.n_rep * L.row_stride_t) + alloc_bytes<float>((size_t)L.n_rep * L.row_stride) +
           2 * alloc_bytes<float2>((size_t)L.Q * L.P * L.C);
  return OAM_OK;
}

}  // namespace

oam_status oam::fft_plan_bytes(const oam_model *m, size_t *bytes) {
  FftLayout L;
  FftPlan pl;
  oam_status rc = fft_plan(m, &L, pl);
  if (rc) return rc;
  return fft_layout_bytes(L, pl, m->grid.nz, bytes);
}

oam_status oam::fft_build(oam_model *m, cudaStream_t st) {
  const int R = m->R, W = m->W, nz = m->grid.nz;
  FftLayout *L = new (std::nothrow) FftLayout();
  if (!L) return OAM_ERR_OOM;
  m->fft = L;
  FftPlan pl;
  {
    oam_status rc0 = fft_plan(m, L, pl);
    if (rc0) return rc0;
  }
  const int P = L->P, Q = L->Q, lgP = L->lgP;
  std::vector<int> &klo = pl.klo, &klen = pl.klen, &rep_of = pl.rep_of;
  std::vector<long long> &koff = pl.koff, &noff = pl.noff;
  std::vector<int2> &krange = pl.krange, &entry_kn = pl.entry_kn;
  std::vector<int4> &members = pl.members;
  oam_status rc;
  if ((rc = dev_alloc(m, &L->d_klo, nz)) || (rc = dev_alloc(m, &L->d_klen, nz)) ||
      (rc = dev_alloc(m, &L->d_koff, nz)) || (rc = dev_alloc(m, &L->d_members, members.size())) ||
      (rc = dev_alloc(m, &L->d_krange, (size_t)L->NS)) || (rc = dev_alloc(m, &L->d_noff, (size_t)L->NS)) ||
      (rc = dev_alloc(m, &L->d_shat_t, (size_t)L->n_rep * L->row_stride_t)) ||
      (rc = dev_alloc(m, &L->d_shat, (size_t)L->n_rep * L->row_stride)) ||
      (rc = dev_alloc(m, &L->d_w1, (size_t)Q * P * L->C)) || (rc = dev_alloc(m, &L->d_w2, (size_t)Q * P * L->C)))
    return rc;
  OAM_CUDA_TRY(cudaMemcpyAsync(L->d_klo, klo.data(), sizeof(int) * nz, cudaMemcpyHostToDevice, st));
  OAM_CUDA_TRY(cudaMemcpyAsync(L->d_klen, klen.data(), sizeof(int) * nz, cudaMemcpyHostToDevice, st));
  OAM_CUDA_TRY(cudaMemcpyAsync(L->d_koff, koff.data(), sizeof(long long) * nz, cudaMemcpyHostToDevice, st));
  OAM_CUDA_TRY(cudaMemcpyAsync(L->d_members, members.data(), sizeof(int4) * members.size(), cudaMemcpyHostToDevice,
                               st));
  OAM_CUDA_TRY(cudaMemcpyAsync(L->d_krange, krange.data(), sizeof(int2) * krange.size(), cudaMemcpyHostToDevice, st));
  OAM_CUDA_TRY(cudaMemcpyAsync(L->d_noff, noff.data(), sizeof(long long) * noff.size(), cudaMemcpyHostToDevice, st));
  // entries of the row by sample whose depth band misses the sample stay zero
  OAM_CUDA_TRY(cudaMemsetAsync(L->d_shat_t, 0, sizeof(float) * (size_t)L->n_rep * L->row_stride_t, st));
  // build S^ (temporaries: entry table, band_hi, rep table, T)
  int2 *d_entry = nullptr;
  int *d_band_hi = nullptr, *d_rep_of = nullptr;
  float *d_T = nullptr;
  const size_t nb = (size_t)m->n_orb * nz;
  if (cudaMallocAsync((void **)&d_entry, sizeof(int2) * entry_kn.size(), st) != cudaSuccess ||
      cudaMallocAsync((void **)&d_band_hi, sizeof(int) * nb, st) != cudaSuccess ||
      cudaMallocAsync((void **)&d_rep_of, sizeof(int) * rep_of.size(), st) != cudaSuccess ||
      cudaMallocAsync((void **)&d_T, sizeof(float) * (size_t)(R + 1) * Q * L->row_len, st) != cudaSuccess) {
    cudaGetLastError();
    if (d_entry) cudaFreeAsync(d_entry, st);
    if (d_band_hi) cudaFreeAsync(d_band_hi, st);
    if (d_rep_of) cudaFreeAsync(d_rep_of, st);
    if (d_T) cudaFreeAsync(d_T, st);
    return OAM_ERR_OOM;
  }
  cudaMemcpyAsync(d_entry, entry_kn.data(), sizeof(int2) * entry_kn.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_band_hi, m->h_band_hi.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_rep_of, rep_of.data(), sizeof(int) * rep_of.size(), cudaMemcpyHostToDevice, st);
  const unsigned eblocks = (unsigned)((L->row_len + kBuildThreads - 1) / kBuildThreads);
  const size_t sb = sizeof(float) * ((size_t)P + (size_t)(R + 1) * kBuildThreads);
  if (sb > 48 * 1024) {
    OAM_CUDA_TRY(cudaFuncSetAttribute(k_shat_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    OAM_CUDA_TRY(cudaFuncSetAttribute(k_shat_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
  }
  k_shat_pass1<<<dim3(eblocks, R + 1), kBuildThreads, sb, st>>>(
      m->d_band, m->d_band_lo, d_band_hi, m->band_w, m->d_tap_orbit, R, W, nz, d_entry, L->row_len, P, Q, d_T);
  OAM_LAUNCHED();
  k_shat_pass2<<<dim3(eblocks, Q), kBuildThreads, sb, st>>>(d_T, L->row_len, R, P, Q, d_rep_of, d_entry, m->n_lo,
                                                            L->d_krange, L->d_noff, L->row_stride, L->row_stride_t, L->d_shat,
                                                            L->d_shat_t);
  OAM_LAUNCHED();
  OAM_CUDA_TRY(cudaStreamSynchronize(st));  // host tables above go out of scope
  cudaFreeAsync(d_entry, st);
  cudaFreeAsync(d_band_hi, st);
  cudaFreeAsync(d_rep_of, st);
  cudaFreeAsync(d_T, st);
  // cost of one application: the banded matrix over all member frequencies
  // (real x complex: 4 flops per entry) and 5 N log2 N per complex transform
  const double half = (double)Q * P;
  const double fft_lines = (double)m->grid.py * m->grid.nz + half / P * m->grid.nz + half / P * L->NS +
                           (double)m->grid.py * L->NS;
  L->flops = 4.0 * half * (double)L->row_len + 5.0 * P * lgP * fft_lines;
  const double c8 = sizeof(float2);
  L->bytes = 4.0 * (double)L->n_rep * L->row_len +                              // S^
             4.0 * vol_elems(m) + 4.0 * (double)m->grid.py * m->grid.px * m->grid.nt +  // input, output
             c8 * Q * m->grid.py * (nz + L->NS) * 2 +                            // row-transform buffers
             c8 * half * (nz + L->NS) * 2;                                       // column-transform buffers
  return OAM_OK;
}

void oam::fft_free(oam_model *m, cudaStream_t st) {
  FftLayout *L = m->fft;
  if (!L) return;
  for (void *p : {(void *)L->d_klo, (void *)L->d_klen, (void *)L->d_koff, (void *)L->d_members, (void *)L->d_krange,
                  (void *)L->d_noff, (void *)L->d_shat_t, (void *)L->d_shat,
                  (void *)L->d_w1, (void *)L->d_w2})
    if (p) cudaFreeAsync(p, st);
  delete L;
  m->fft = nullptr;
}

double oam::fft_flops(const oam_model *m) { return m->fft ? m->fft->flops : 0.0; }
double oam::fft_bytes(const oam_model *m) { return m->fft ? m->fft->bytes : 0.0; }

namespace {

oam_status set_smem(const void *fn, size_t bytes) {
  if (bytes > 48 * 1024)
    OAM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return OAM_OK;
}

}  // namespace

namespace {

// Threads for a register-pass transform block: one per group of the
// four-stage passes (KL lines x P/16 groups), 64 to 256.
int xthreads(int P, int KL) { return std::max(64, std::min(kFftThreads, (((P >> 4) * KL + 31) / 32) * 32)); }

// The transforms of one application in register passes (P >= 16); the
// spectral products are launched by run_fft between them.
template <int KC>
struct XKernels {
  static oam_status prepare(int P) {
    oam_status rc;
    const size_t sr = sizeof(float2) * xslots<KC / 2>(P), sc = sizeof(float2) * xslots<KC>(P);
    if ((rc = set_smem((const void *)k_xfft_rows_r2c<KC>, sr)) || (rc = set_smem((const void *)k_xfft_rows_c2r<KC>, sr)) ||
        (rc = set_smem((const void *)k_xfft_cols<KC, false>, sc)) || (rc = set_smem((const void *)k_xfft_cols<KC, true>, sc)))
      return rc;
    return OAM_OK;
  }
  static void rows_r2c(dim3 g, cudaStream_t st, const float *X, int py, int px, int Ctot, int c0, int C, int P, int lgP,
                       int Q, float2 *Y) {
    k_xfft_rows_r2c<KC><<<g, xthreads(P, KC / 2), sizeof(float2) * xslots<KC / 2>(P), st>>>(X, py, px, Ctot, c0, C, P,
                                                                                           lgP, Q, Y);
  }
  static void cols(dim3 g, cudaStream_t st, const float2 *Z, int nin, int nout, int C, int P, int lgP, int inverse,
                   float2 *W) {
    if (inverse)
      k_xfft_cols<KC, true><<<g, xthreads(P, KC), sizeof(float2) * xslots<KC>(P), st>>>(Z, nin, nout, C, P, lgP, W);
    else
      k_xfft_cols<KC, false><<<g, xthreads(P, KC), sizeof(float2) * xslots<KC>(P), st>>>(Z, nin, nout, C, P, lgP, W);
  }
  static void rows_c2r(dim3 g, cudaStream_t st, const float2 *Z, int py, int px, int Ctot, int c0, int C, int P,
                       int lgP, int Q, float scale, float *X) {
    k_xfft_rows_c2r<KC><<<g, xthreads(P, KC / 2), sizeof(float2) * xslots<KC / 2>(P), st>>>(Z, py, px, Ctot, c0, C,
                                                                                           P, lgP, Q, scale, X);
  }
};

// The same in the radix-2 kernels (any P).
template <int KC>
struct RKernels {
  static oam_status prepare(int P) {
    oam_status rc;
    const size_t sm = fft_smem(P, KC), smr = fft_smem(P, KC / 2);  // row kernels: two channels per line
    if ((rc = set_smem((const void *)k_fft_rows_r2c<KC>, smr)) || (rc = set_smem((const void *)k_fft_cols<KC>, sm)) ||
        (rc = set_smem((const void *)k_fft_rows_c2r<KC>, smr)))
      return rc;
    return OAM_OK;
  }
  static void rows_r2c(dim3 g, cudaStream_t st, const float *X, int py, int px, int Ctot, int c0, int C, int P, int lgP,
                       int Q, float2 *Y) {
    k_fft_rows_r2c<KC><<<g, kFftThreads, fft_smem(P, KC / 2), st>>>(X, py, px, Ctot, c0, C, P, lgP, Q, Y);
  }
  static void cols(dim3 g, cudaStream_t st, const float2 *Z, int nin, int nout, int C, int P, int lgP, int inverse,
                   float2 *W) {
    k_fft_cols<KC><<<g, kFftThreads, fft_smem(P, KC), st>>>(Z, nin, nout, C, P, lgP, inverse, W);
  }
  static void rows_c2r(dim3 g, cudaStream_t st, const float2 *Z, int py, int px, int Ctot, int c0, int C, int P,
                       int lgP, int Q, float scale, float *X) {
    k_fft_rows_c2r<KC><<<g, kFftThreads, fft_smem(P, KC / 2), st>>>(Z, py, px, Ctot, c0, C, P, lgP, Q, scale, X);
  }
};

template <int KC, class K>
oam_status run_fft(const oam_model *m, const FftLayout *L, bool fwd, const float *in, float *out, cudaStream_t st) {
  const int P = L->P, Q = L->Q, lgP = L->lgP, nz = m->grid.nz, py = m->grid.py, px = m->grid.px, NS = L->NS;
  oam_status rc = K::prepare(P);
  if (rc) return rc;
  const unsigned cbz = (unsigned)((nz + KC - 1) / KC), cbs = (unsigned)((NS + KC - 1) / KC);
  const float scale = 1.0f / ((float)P * (float)P);
  if (fwd) {
    K::rows_r2c(dim3(py, cbz), st, in, py, px, nz, 0, nz, P, lgP, Q, L->d_w2);
    OAM_LAUNCHED();
    K::cols(dim3(Q, cbz), st, L->d_w2, py, P, nz, P, lgP, 0, L->d_w1);
    OAM_LAUNCHED();
    const size_t sa = sizeof(float4) * 2 * nz + sizeof(int) * (2 * nz + 2) + sizeof(long long) * nz;
    if ((rc = set_smem((const void *)k_fft_apply_fwd, sa))) return rc;
    const int fchunk = kFwdChunk > 0 ? kFwdChunk : NS;
    const int fwd_threads = std::min(kApplyMaxThreads, 32 * ((fchunk + 32 / kFwdPhases - 1) / (32 / kFwdPhases)));
    const unsigned fblocks = (unsigned)(L->n_rep * ((NS + fchunk - 1) / fchunk));
    k_fft_apply_fwd<<<fblocks, fwd_threads, sa, st>>>(L->d_shat, L->row_stride, L->d_members, L->d_klo, L->d_klen,
                                                      L->d_koff, L->d_krange, nz, m->n_lo, NS, L->d_w1, L->d_w2);
    OAM_LAUNCHED();
    K::cols(dim3(Q, cbs), st, L->d_w2, P, py, NS, P, lgP, 1, L->d_w1);
    OAM_LAUNCHED();
    const unsigned cbt = (unsigned)((m->grid.nt + KC - 1) / KC);
    K::rows_c2r(dim3(py, cbt), st, L->d_w1, py, px, m->grid.nt, m->n_lo, NS, P, lgP, Q, scale, out);
    OAM_LAUNCHED();
  } else {
    K::rows_r2c(dim3(py, cbs), st, in, py, px, m->grid.nt, m->n_lo, NS, P, lgP, Q, L->d_w2);
    OAM_LAUNCHED();
    K::cols(dim3(Q, cbs), st, L->d_w2, py, P, NS, P, lgP, 0, L->d_w1);
    OAM_LAUNCHED();
    const size_t sa = (sizeof(float4) * 2 + sizeof(int2) + sizeof(long long)) * NS;
    if ((rc = set_smem((const void *)k_fft_apply_adj, sa))) return rc;
    const int achunk = kAdjChunk > 0 ? kAdjChunk : nz;
    const int adj_threads = std::min(kApplyMaxThreads, 32 * ((achunk + 15) / 16));
    const unsigned ablocks = (unsigned)(L->n_rep * ((nz + achunk - 1) / achunk));
    k_fft_apply_adj<<<ablocks, adj_threads, sa, st>>>(L->d_shat_t, L->row_stride_t, L->d_members, L->d_klo, L->d_klen,
                                                      L->d_krange, L->d_noff, nz, m->n_lo, NS, L->d_w1, L->d_w2);
    OAM_LAUNCHED();
    K::cols(dim3(Q, cbz), st, L->d_w2, P, py, nz, P, lgP, 1, L->d_w1);
    OAM_LAUNCHED();
    K::rows_c2r(dim3(py, cbz), st, L->d_w1, py, px, nz, 0, nz, P, lgP, Q, scale, out);
    OAM_LAUNCHED();
  }
  return OAM_OK;
}

oam_status run_fft_any(const oam_model *m, bool fwd, const float *in, float *out, cudaStream_t st) {
  const FftLayout *L = m->fft;
  if (!L) return OAM_ERR_UNSUPPORTED;
  ProfScope prof(m, st, fwd);
  const bool x = L->P >= 16;  // register-pass transforms need a four-stage pass
  switch (L->KC) {
    case 16: return x ? run_fft<16, XKernels<16>>(m, L, fwd, in, out, st) : run_fft<16, RKernels<16>>(m, L, fwd, in, out, st);
    case 8: return x ? run_fft<8, XKernels<8>>(m, L, fwd, in, out, st) : run_fft<8, RKernels<8>>(m, L, fwd, in, out, st);
    case 4: return x ? run_fft<4, XKernels<4>>(m, L, fwd, in, out, st) : run_fft<4, RKernels<4>>(m, L, fwd, in, out, st);
    default: return x ? run_fft<2, XKernels<2>>(m, L, fwd, in, out, st) : run_fft<2, RKernels<2>>(m, L, fwd, in, out, st);
  }
}

}  // namespace

oam_status oam::forward_fft(const oam_model *m, const float *H, float *s, cudaStream_t st) {
  return run_fft_any(m, true, H, s, st);
}

oam_status oam::adjoint_fft(const oam_model *m, const float *s, float *H, cudaStream_t st) {
  return run_fft_any(m, false, s, H, st);
}
