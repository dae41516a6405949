// Model slab builder (Methods, Forward modeling, Eqs. 1-4): per-orbit bands
// of the single-position model, and the FP32 operator layouts packed from them.
//
// Distances use the cancellation-free form d - F = (2F r.n + |r|^2) / (d + F)
// in FP64, so the arrival sample fs*(d/c - t0) = (fs/c)(d - F) + fs(F/c - t0)
// keeps full precision; the EIR derivative is evaluated in FP32 at
// tau = n - D_j (|tau| <= trunc_sigma * sigma_s), tau being the FP32 rounding
// of the exact offset, and summed over patches with a compensated FP32 sum.
#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.cuh"

using namespace oam;

namespace {

struct Geo {
  double F, dx, dy, dz, z0;
  double ks;      // fs / c, samples per metre
  double G;       // fs * (F/c - t0)
  double cut;     // truncation, samples
  float inv2s2;   // 1 / (2 sigma_s^2)
  float env2;     // log2(e) / (2 sigma_s^2): envelope exp(-tau^2 / (2 sigma_s^2)) = 2^(-env2 tau^2)
  float invs2;    // 1 / sigma_s^2
  float omega;    // 2 pi fc / fs
  float cyc;      // 2 fc / fs: the phase omega * tau in units of pi
};

// d - F for the voxel at lateral offset (a dx, b dy), depth k, and patch normal n.
__device__ __forceinline__ double delta_dist(const Geo &g, int b, int a, int k, Patch p) {
  double rx = a * g.dx, ry = b * g.dy, rz = g.z0 + k * g.dz;
  double rn = __dadd_rn(__dadd_rn(__dmul_rn(rx, p.x), __dmul_rn(ry, p.y)), __dmul_rn(rz, p.z));
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
  double num = __dadd_rn(__dmul_rn(2.0 * g.F, rn), r2);
  double d = sqrt(__dadd_rn(__dmul_rn(g.F, g.F), num));
  return __ddiv_rn(num, __dadd_rn(d, g.F));
}

// ---------------------------------------------------------------- double-word FP32
// A pair (h, l) of floats with |l| <= ulp(h)/2 carries about 48 significand
// bits, enough for patch arrivals to 1e-11 samples, at FP32 instruction rates
// (this GPU's FP64 rate is far lower).  Error-free transforms and the add,
// multiply, divide and square-root steps follow Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 2017); the _rn intrinsics keep the compiler from
// contracting or reordering them.
struct DW {
  float h, l;
};
__device__ __forceinline__ DW fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DW two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), ap = __fsub_rn(s, b), bp = __fsub_rn(s, ap);
  return {s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp))};
}
__device__ __forceinline__ DW two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DW dw_add(DW x, DW y) {
  const DW s = two_sum(x.h, y.h), t = two_sum(x.l, y.l);
  const DW v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}
__device__ __forceinline__ DW dw_mul(DW x, DW y) {
  const DW c = two_prod(x.h, y.h);
  const float t = __fmaf_rn(x.l, y.h, __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.l)));
  return fast_two_sum(c.h, __fadd_rn(c.l, t));
}
__device__ __forceinline__ DW dw_mul_f(DW x, float y) {
  const DW c = two_prod(x.h, y);
  const DW t = fast_two_sum(c.h, __fmul_rn(x.l, y));
  return fast_two_sum(t.h, __fadd_rn(t.l, c.l));
}
__device__ __forceinline__ DW dw_div(DW x, DW y) {
  const float th = __fdiv_rn(x.h, y.h);
  const DW r = dw_mul_f(y, th);
  const float d = __fadd_rn(__fsub_rn(x.h, r.h), __fsub_rn(x.l, r.l));
  return fast_two_sum(th, __fdiv_rn(d, y.h));
}
__device__ __forceinline__ DW dw_sqrt(DW x) {  // x > 0: one Newton step from the FP32 root
  const float s = __fsqrt_rn(x.h);
  const float e = __fadd_rn(__fmaf_rn(-s, s, x.h), x.l);
  return fast_two_sum(s, __fdiv_rn(e, __fmul_rn(2.0f, s)));
}
__device__ __forceinline__ DW to_dw(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

// Patch normal as double words and weight in mm^2 per metre of distance.
struct __align__(32) PatchDW {
  float xh, xl, yh, yl, zh, zl, w, pad;
};

__global__ void k_patch_dw(const Patch *__restrict__ patch, int M, PatchDW *__restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    const Patch p = patch[j];
    const DW x = to_dw(p.x), y = to_dw(p.y), z = to_dw(p.z);
    out[j] = PatchDW{x.h, x.l, y.h, y.l, z.h, z.l, (float)(p.w * 1e-3), 0.0f};
  }
}

// d - F in plain FP32 (same cancellation-free form).  Its error is below
// 4e-7 |r|, r the voxel offset (|d - F| <= |r|).
__device__ __forceinline__ float delta_dist_f(float rx, float ry, float rz, float r2, float F, const PatchDW &p) {
  const float rn = rx * p.xh + ry * p.yh + rz * p.zh;
  const float num = 2.0f * F * rn + r2;
  const float d = sqrtf(F * F + num);
  return num / (d + F);
}

template <bool kMax>
__device__ __forceinline__ float block_ext(float v, float *sh) {
  for (int off = 16; off; off >>= 1) {
    const float o = __shfl_xor_sync(0xffffffffu, v, off);
    v = kMax ? fmaxf(v, o) : fminf(v, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = sh[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) v = kMax ? fmaxf(v, sh[i]) : fminf(v, sh[i]);
  return v;
}

// Per (orbit, depth): min and max of d - F over the patches, exactly as FP64
// evaluates them.  Plain FP32 distances locate the extremes; only patches
// within 1e-5 |r| of the FP32 extremes (a bound 25x the FP32 error) are
// evaluated in FP64, so the true FP64 extremes are always among them.
__global__ void k_delta_range(Geo g, const Patch *__restrict__ patch, const PatchDW *__restrict__ pdw, int M,
                              const int *orb_b, const int *orb_a, int nz, double2 *out) {
  __shared__ float shf[32];
  __shared__ double slo[32], shi[32];
  const int o = blockIdx.x, k = blockIdx.y;
  const int b = orb_b[o], a = orb_a[o];
  const double rxd = a * g.dx, ryd = b * g.dy, rzd = g.z0 + k * g.dz;
  const float rx = (float)rxd, ry = (float)ryd, rz = (float)rzd;
  const float r2 = (float)(rxd * rxd + ryd * ryd + rzd * rzd), F = (float)g.F;
  float lo32 = INFINITY, hi32 = -INFINITY;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const float dd = delta_dist_f(rx, ry, rz, r2, F, pdw[j]);
    lo32 = fminf(lo32, dd);
    hi32 = fmaxf(hi32, dd);
  }
  lo32 = block_ext<false>(lo32, shf);
  hi32 = block_ext<true>(hi32, shf);
  const float tol = 1e-5f * sqrtf(r2);
  double lo = INFINITY, hi = -INFINITY;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const float dd = delta_dist_f(rx, ry, rz, r2, F, pdw[j]);
    if (dd <= lo32 + tol || dd >= hi32 - tol) {
      const double d64 = delta_dist(g, b, a, k, patch[j]);
      if (dd <= lo32 + tol) lo = fmin(lo, d64);
      if (dd >= hi32 - tol) hi = fmax(hi, d64);
    }
  }
  for (int off = 16; off; off >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    slo[w] = lo;
    shi[w] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      lo = fmin(lo, slo[i]);
      hi = fmax(hi, shi[i]);
    }
    out[o * nz + k] = make_double2(lo, hi);
  }
}

// ---------------------------------------------------------------- trilinear voxels
// The paper's discretisation of Eq. 1 (Methods, Forward modeling): the
// surface integral of the trilinear interpolation of the voxel values, and a
// central finite difference in time.  A voxel is the tent
// L(x/dx) L(y/dy) L(z/dz), L(u) = max(0, 1 - |u|); across its support the
// sphere |x - x'| = ct is a plane, so the integral is the tent's planar
// Radon transform along e = (v - q)/|v - q|: the hats of half-width
// a = |e_i| d_i (area d_i) convolve, i.e. a six-box spline
//   sum over sign vectors s of prod(s) (u + sum s_i c_i/2)_+^5 / 5!,
// with an axis whose a < 1e-3 max(a) taken as a spike of mass d_i.  FP64:
// the signed sum cancels heavily.
__device__ double tent_radon(double dx, double dy, double dz, double ex, double ey, double ez, double u) {
  const double d[3] = {dx, dy, dz}, e[3] = {fabs(ex), fabs(ey), fabs(ez)};
  double a[3], amax = 0.0;
  for (int i = 0; i < 3; ++i) {
    a[i] = e[i] * d[i];
    amax = fmax(amax, a[i]);
  }
  double c[6], scale = 1.0;
  int n = 0;
  for (int i = 0; i < 3; ++i) {
    if (a[i] < 1e-3 * amax) {
      scale *= d[i];
    } else {
      c[n++] = a[i];
      c[n++] = a[i];
      scale *= d[i] / (a[i] * a[i]);
    }
  }
  double fact = 1.0;
  for (int i = 2; i < n; ++i) fact *= i;
  double sum = 0.0;
  for (int mask = 0; mask < (1 << n); ++mask) {
    double x = u, sign = 1.0;
    for (int i = 0; i < n; ++i) {
      if (mask & (1 << i)) {
        x -= 0.5 * c[i];
        sign = -sign;
      } else {
        x += 0.5 * c[i];
      }
    }
    if (x > 0.0) {
      double pw = 1.0;
      for (int q = 1; q < n; ++q) pw *= x;
      sum += sign * pw;
    }
  }
  return scale * sum / fact;
}

struct Geo33 {
  double F, dx, dy, dz, z0;  // mm
  double c;                  // mm / s
  double fs, t0;             // Hz, s
  double sigma, omega;       // EIR in samples: std dev, rad per sample
  int T;                     // EIR taps each side (whole samples within the cut)
  int len;                   // samples of a patch's finite-difference support held per patch
};

constexpr int k33Chunk = 128;  // patches per shared-memory chunk

// Block (orbit o, depth k): band values S[o][k][lo .. hi) =
//   sum_j w_j sum_m e(n - m) D_j(m),  D_j(m) = (I_j(m+1) - I_j(m-1)) / 2,
//   I_j(m) = R_j(c t_m - r_j) / (c t_m),  t_m = t0 + m / fs,
// patches in index order, each patch's sum over m first (FP64 throughout).
__global__ void k_slab33_values(Geo33 g, const Patch *__restrict__ patch, int M, const int *orb_b, const int *orb_a,
                                int nz, int nt, const int *band_lo, const int *band_hi, int band_w,
                                float *__restrict__ band) {
  extern __shared__ double sm33[];
  double *e = sm33;                           // [2T + 1]
  double *D = e + 2 * g.T + 1;                // [k33Chunk][len]
  int *m0s = reinterpret_cast<int *>(D + (size_t)k33Chunk * g.len);  // [k33Chunk]
  double *ws = reinterpret_cast<double *>(m0s + k33Chunk + (k33Chunk & 1));  // [k33Chunk] (8-byte aligned)
  const int o = blockIdx.x, k = blockIdx.y;
  const double vx = orb_a[o] * g.dx, vy = orb_b[o] * g.dy, vz = g.z0 + k * g.dz;
  const int lo = band_lo[(size_t)o * nz + k], hi = band_hi[(size_t)o * nz + k];
  for (int i = threadIdx.x; i <= 2 * g.T; i += blockDim.x) {
    const double tau = i - g.T;
    e[i] = exp(-tau * tau / (2.0 * g.sigma * g.sigma)) * cos(g.omega * tau);
  }
  constexpr int kPer = 4;  // band samples per thread (band_w <= 4 * blockDim)
  double acc[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) acc[q] = 0.0;
  const double h = g.dx + g.dy + g.dz;
  for (int j0 = 0; j0 < M; j0 += k33Chunk) {
    __syncthreads();
    for (int i = threadIdx.x; i < k33Chunk; i += blockDim.x) {
      const int j = j0 + i;
      if (j >= M) {
        m0s[i] = INT_MIN / 2;
        continue;
      }
      const Patch pj = patch[j];
      const double ux = vx + g.F * pj.x, uy = vy + g.F * pj.y, uz = vz + g.F * pj.z;  // v - q, q = -F n
      const double r = sqrt(ux * ux + uy * uy + uz * uz);
      const double ex = ux / r, ey = uy / r, ez = uz / r;
      const int m0 = (int)floor(g.fs * ((r - h) / g.c - g.t0)) - 1;
      m0s[i] = m0;
      ws[i] = pj.w;
      for (int q = 0; q < g.len; ++q) {
        const int m = m0 + q;
        double dv = 0.0;
        if (m >= -1 && m <= nt) {
          const double rho1 = g.c * (g.t0 + (m + 1) / g.fs), rho0 = g.c * (g.t0 + (m - 1) / g.fs);
          const double i1 = tent_radon(g.dx, g.dy, g.dz, ex, ey, ez, rho1 - r) / rho1;
          const double i0 = tent_radon(g.dx, g.dy, g.dz, ex, ey, ez, rho0 - r) / rho0;
          dv = 0.5 * (i1 - i0);
        }
        D[(size_t)i * g.len + q] = dv;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int n = lo + threadIdx.x + q * blockDim.x;
      if (n >= hi) continue;
      for (int i = 0; i < k33Chunk; ++i) {
        const int m0 = m0s[i];
        if (n < m0 - g.T || n > m0 + g.len - 1 + g.T) continue;
        double sj = 0.0;
        for (int qq = 0; qq < g.len; ++qq) {
          const int dm = n - (m0 + qq);
          if (dm >= -g.T && dm <= g.T) sj += e[dm + g.T] * D[(size_t)i * g.len + qq];
        }
        acc[q] += ws[i] * sj;
      }
    }
  }
  float *row = band + ((size_t)o * nz + k) * band_w;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = threadIdx.x + q * blockDim.x;
    if (i < band_w) row[i] = lo + i < hi ? (float)acc[q] : 0.0f;
  }
}

constexpr int kPatchChunk = 512;

// Band values: thread i of block (o, k) owns sample lo + i (+ blockDim.x ...).
// Each patch's arrival D = (fs/c)(d - F) + fs(F/c - t0) (samples, double-word
// FP32, ~1e-11 samples) is split into the nearest sample n_ref and a fraction
// f = D - n_ref in [-1/2, 1/2], so tau = (n - n_ref) - f is the FP32 rounding
// of the offset.  The phase omega*tau is a rotation: the patch's own
// (cos, sin)(-omega f) turned by a table entry (cos, sin)(omega t) for the
// integer t = n - n_ref (|t| <= cut + 1/2); both arguments are small, so the
// result stays within a few ulp.  The envelope is exp2 of a pre-scaled
// argument and the patch sum is a compensated (Kahan) FP32 sum.  Patches are
// visited in index order, so every entry is a fixed-order sum.
__global__ void k_slab_values(Geo g, const PatchDW *__restrict__ pdw, int M, const int *orb_b,
                              const int *orb_a, int nz, const int *band_lo, const int *band_hi,
                              int band_w, int T0, float *band) {
  extern __shared__ float2 rot[];  // [2 T0 + 1]: (cos, sin)(omega t), t = -T0 .. T0
  const int o = blockIdx.x, k = blockIdx.y;
  const int b = orb_b[o], a = orb_a[o];
  const int lo = band_lo[o * nz + k], hi = band_hi[o * nz + k];
  __shared__ float4 sP[kPatchChunk];  // (n_ref, f, cos(omega f), -sin(omega f))
  __shared__ float sW[kPatchChunk];
  for (int t = threadIdx.x; t <= 2 * T0; t += blockDim.x) {
    float sn, cs;
    sincospif(g.cyc * (float)(t - T0), &sn, &cs);
    rot[t] = make_float2(cs, sn);
  }
  const int per = (band_w + blockDim.x - 1) / blockDim.x;  // samples per thread (<= 4)
  const float cut = (float)g.cut;
  float sum[4] = {0, 0, 0, 0}, comp[4] = {0, 0, 0, 0};
  // block constants as double words (voxel offset, |r|^2, F, 2F, F^2, fs/c, G)
  const double rxd = a * g.dx, ryd = b * g.dy, rzd = g.z0 + k * g.dz;
  const DW rx = to_dw(rxd), ry = to_dw(ryd), rz = to_dw(rzd), r2 = to_dw(rxd * rxd + ryd * ryd + rzd * rzd);
  const DW Fw = to_dw(g.F), F2w = to_dw(2.0 * g.F), FFw = to_dw(g.F * g.F), ks = to_dw(g.ks), G = to_dw(g.G);
  for (int j0 = 0; j0 < M; j0 += kPatchChunk) {
    const int cnt = min(kPatchChunk, M - j0);
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const PatchDW p = pdw[j0 + j];
      const DW rn = dw_add(dw_add(dw_mul(rx, DW{p.xh, p.xl}), dw_mul(ry, DW{p.yh, p.yl})), dw_mul(rz, DW{p.zh, p.zl}));
      const DW num = dw_add(dw_mul(F2w, rn), r2);
      const DW d = dw_sqrt(dw_add(FFw, num));
      const DW dd = dw_div(num, dw_add(d, Fw));        // d - F, metres
      const DW D = dw_add(dw_mul(ks, dd), G);           // arrival, samples
      const float nr = rintf(D.h);
      const float f = __fadd_rn(__fsub_rn(D.h, nr), D.l);  // D.h - nr is exact
      float sn, cs;
      sincospif(g.cyc * f, &sn, &cs);
      sP[j] = make_float4(nr, f, cs, -sn);
      sW[j] = __fdiv_rn(p.w, dw_add(Fw, dd).h);         // (mm^2 / 1e3) / metres = mm^2 / mm
    }
    __syncthreads();
    for (int r = 0; r < per; ++r) {
      const int n = lo + threadIdx.x + r * blockDim.x;
      if (n >= hi) break;
      const float nf = (float)n;
      float s = sum[r], c = comp[r];
      for (int j = 0; j < cnt; ++j) {
        const float4 q = sP[j];
        const float t = nf - q.x;  // exact integer
        const float tau = t - q.y;
        if (fabsf(tau) <= cut) {
          const float2 e = rot[__float2int_rn(t) + T0];  // |t| <= cut + 1/2 < T0
          const float cs = e.x * q.z - e.y * q.w;        // cos(omega t - omega f)
          const float sn = e.y * q.z + e.x * q.w;        // sin(omega t - omega f)
          const float env = exp2f(-tau * tau * g.env2);
          const float v = -env * (tau * g.invs2 * cs + g.omega * sn);
          const float y = sW[j] * v - c;
          const float u = s + y;
          c = (u - s) - y;
          s = u;
        }
      }
      sum[r] = s;
      comp[r] = c;
    }
  }
  float *row = band + ((size_t)o * nz + k) * band_w;
  for (int r = 0; r < per; ++r) {
    const int i = threadIdx.x + r * blockDim.x;
    if (i >= band_w) break;
    const int n = lo + i;
    row[i] = (n < hi) ? sum[r] - comp[r] : 0.0f;
  }
}

// FP32 forward layout: rows k in [klo, khi) of kTimeTile samples of tile T.
__global__ void k_pack_fwd(const float *band, const int *band_lo, const int *band_hi, int band_w, int nz,
                           int n_ttiles, const int *krange, const long long *off, float *out) {
  const int ot = blockIdx.x;
  const int o = ot / n_ttiles, T = ot % n_ttiles;
  const int klo = krange[2 * ot], khi = krange[2 * ot + 1];
  const long long base = off[ot];
  const int total = (khi - klo) * kTimeTile;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int k = klo + i / kTimeTile, n = T * kTimeTile + i % kTimeTile;
    const int lo = band_lo[o * nz + k], hi = band_hi[o * nz + k];
    out[base + i] = (n >= lo && n < hi) ? band[((size_t)o * nz + k) * band_w + (n - lo)] : 0.0f;
  }
}

// FP32 adjoint layout: kDepthTile rows (depths) of nlen samples from nlo.
__global__ void k_pack_adj(const float *band, const int *band_lo, const int *band_hi, int band_w, int nz,
                           int n_ktiles, const int *nrange, const long long *off, float *out) {
  const int ok = blockIdx.x;
  const int o = ok / n_ktiles, K = ok % n_ktiles;
  const int nlo = nrange[2 * ok], nlen = nrange[2 * ok + 1];
  const long long base = off[ok];
  const int total = kDepthTile * nlen;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int k = K * kDepthTile + i / nlen, n = nlo + i % nlen;
    float v = 0.0f;
    if (k < nz) {
      const int lo = band_lo[o * nz + k], hi = band_hi[o * nz + k];
      if (n >= lo && n < hi) v = band[((size_t)o * nz + k) * band_w + (n - lo)];
    }
    out[base + i] = v;
  }
}

__global__ void k_slab_column(const float *band, const int *band_lo, int band_w, int nz, int nt, int o, int k,
                              float *out) {
  const int lo = band_lo[o * nz + k];
  const float *row = band + ((size_t)o * nz + k) * band_w;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nt; n += gridDim.x * blockDim.x) {
    const int i = n - lo;
    out[n] = (i >= 0 && i < band_w) ? row[i] : 0.0f;
  }
}

}  // namespace

int oam::disc_margin(const oam_model *m) {
  if (m->disc != OAM_DISC_TRILINEAR) return 0;
  const oam_grid &g = m->grid;
  return (int)std::ceil(g.fs_hz * (g.dx_m + g.dy_m + g.dz_m) / m->sensor.c_mps) + 2;
}

// Time origin, window check and bands [lo, hi) per (orbit, depth) from the
// range of d - F over the patches; each band is widened by `widen` samples on
// both sides (0 for a model build; the footprint planner widens to cover
// rounding of its host-side distances).  Also the slab's nonzero count and
// the operator's algorithmic flops.
oam_status oam::plan_bands(oam_model *m, const std::vector<double2> &h_range, int widen) {
  const oam_grid &gr = m->grid;
  const int nz = gr.nz, nt = gr.nt, O = m->n_orb;
  double dmin = INFINITY, dmax = -INFINITY;
  for (const double2 &r : h_range) {
    dmin = std::min(dmin, r.x);
    dmax = std::max(dmax, r.y);
  }
  const double fs = gr.fs_hz, c = m->sensor.c_mps, F = m->sensor.focal_m, ks = fs / c;
  const double reach = m->cut + disc_margin(m);  // samples an arrival reaches on either side
  const double t0 = std::isnan(gr.t0_s) ? (std::floor(fs * (F + dmin) / c - reach) - 2.0) / fs : gr.t0_s;
  m->t0 = t0;
  const double G = fs * (F / c - t0);
  if (ks * dmin + G - reach < 0 || ks * dmax + G + reach >= nt) return OAM_ERR_WINDOW;
  m->G = G;
  widen += disc_margin(m);

  // bands [lo, hi) per (orbit, depth)
  m->h_band_lo.resize((size_t)O * nz);
  m->h_band_hi.resize((size_t)O * nz);
  int wmax = 1;
  m->n_lo = nt;
  m->n_hi = 0;
  for (size_t i = 0; i < h_range.size(); ++i) {
    int lo = (int)std::ceil(ks * h_range[i].x + G - m->cut) - widen;
    int hi = (int)std::floor(ks * h_range[i].y + G + m->cut) + 1 + widen;
    lo = std::max(lo, 0);
    hi = std::min(hi, nt);
    if (hi < lo) hi = lo;
    m->h_band_lo[i] = lo;
    m->h_band_hi[i] = hi;
    wmax = std::max(wmax, hi - lo);
    if (hi > lo) {
      m->n_lo = std::min(m->n_lo, lo);
      m->n_hi = std::max(m->n_hi, hi);
    }
  }
  m->band_w = (wmax + 3) & ~3;
  if (m->band_w > 512) return OAM_ERR_UNSUPPORTED;

  // algorithmic work: entries in bands, and multiply-adds over in-grid voxel/position pairs
  std::vector<long long> orb_sum(O, 0);
  for (int o = 0; o < O; ++o)
    for (int k = 0; k < nz; ++k) orb_sum[o] += m->h_band_hi[(size_t)o * nz + k] - m->h_band_lo[(size_t)o * nz + k];
  long long nnz = 0;
  double fl = 0;
  for (int b = -m->R; b <= m->R; ++b)
    for (int a = -m->R; a <= m->R; ++a) {
      long long sum = orb_sum[m->h_tap_orbit[(b + m->R) * m->W + (a + m->R)]];
      nnz += sum;
      long long pairs = (long long)std::max(0, gr.py - std::abs(b)) * std::max(0, gr.px - std::abs(a));
      fl += 2.0 * (double)pairs * (double)sum;
    }
  m->nnz = nnz;
  m->flops = fl;
  return OAM_OK;
}

// FP32 forward layout: per (orbit, 64-sample time tile) the depths [klo, khi)
// whose band meets the tile, rows of kTimeTile samples.  Returns the floats.
long long oam::fwd_layout(const oam_model *m, std::vector<int> *kr, std::vector<long long> *off) {
  const int nz = m->grid.nz, O = m->n_orb, NT = (m->grid.nt + kTimeTile - 1) / kTimeTile;
  kr->assign((size_t)O * NT * 2, 0);
  off->assign((size_t)O * NT, 0);
  long long total = 0;
  for (int o = 0; o < O; ++o)
    for (int T = 0; T < NT; ++T) {
      int klo = nz, khi = 0;
      for (int k = 0; k < nz; ++k) {
        int lo = m->h_band_lo[(size_t)o * nz + k], hi = m->h_band_hi[(size_t)o * nz + k];
        if (hi > lo && lo < (T + 1) * kTimeTile && hi > T * kTimeTile) {
          klo = std::min(klo, k);
          khi = std::max(khi, k + 1);
        }
      }
      if (khi <= klo) klo = khi = 0;
      size_t i = (size_t)o * NT + T;
      (*kr)[2 * i] = klo;
      (*kr)[2 * i + 1] = khi;
      (*off)[i] = total;
      total += (long long)(khi - klo) * kTimeTile;
    }
  return total;
}

// FP32 adjoint layout: per (orbit, 16-depth tile) the union sample range
// [nlo, nlo + nlen), 4-aligned, rows of nlen samples.  Returns the floats.
long long oam::adj_layout(const oam_model *m, std::vector<int> *nr, std::vector<long long> *off) {
  const int nz = m->grid.nz, nt = m->grid.nt, O = m->n_orb, NK = (nz + kDepthTile - 1) / kDepthTile;
  nr->assign((size_t)O * NK * 2, 0);
  off->assign((size_t)O * NK, 0);
  long long total = 0;
  for (int o = 0; o < O; ++o)
    for (int K = 0; K < NK; ++K) {
      int nlo = nt, nhi = 0;
      for (int k = K * kDepthTile; k < std::min(nz, (K + 1) * kDepthTile); ++k) {
        int lo = m->h_band_lo[(size_t)o * nz + k], hi = m->h_band_hi[(size_t)o * nz + k];
        if (hi > lo) {
          nlo = std::min(nlo, lo);
          nhi = std::max(nhi, hi);
        }
      }
      if (nhi <= nlo) {
        nlo = 0;
        nhi = 0;
      }
      nlo &= ~3;
      nhi = std::min((nhi + 3) & ~3, nt);
      size_t i = (size_t)o * NK + K;
      (*nr)[2 * i] = nlo;
      (*nr)[2 * i + 1] = nhi - nlo;
      (*off)[i] = total;
      total += (long long)kDepthTile * (nhi - nlo);
    }
  return total;
}

// Device bytes build_slab allocates for a model whose bands are planned.
size_t oam::slab_plan_bytes(const oam_model *m) {
  const size_t O = m->n_orb, nz = m->grid.nz;
  std::vector<int> iv;
  std::vector<long long> lv;
  const size_t NT = (m->grid.nt + kTimeTile - 1) / kTimeTile, NK = (nz + kDepthTile - 1) / kDepthTile;
  size_t b = alloc_bytes<int>((size_t)m->W * m->W) + alloc_bytes<int>(O * nz) + alloc_bytes<float>(O * nz * m->band_w);
  b += alloc_bytes<int>(O * NT * 2) + alloc_bytes<long long>(O * NT) + alloc_bytes<float>(fwd_layout(m, &iv, &lv));
  b += alloc_bytes<int>(O * NK * 2) + alloc_bytes<long long>(O * NK) + alloc_bytes<float>(adj_layout(m, &iv, &lv));
  return b;
}

oam_status oam::build_slab(oam_model *m, cudaStream_t st) {
  const oam_grid &gr = m->grid;
  const int nz = gr.nz, nt = gr.nt, O = m->n_orb;
  oam_status rc;
  int *d_orb_b = nullptr, *d_orb_a = nullptr;
  double2 *d_range = nullptr;
  if ((rc = dev_alloc(m, &m->d_tap_orbit, m->W * m->W))) return rc;
  OAM_CUDA_TRY(cudaMemcpyAsync(m->d_tap_orbit, m->h_tap_orbit.data(), sizeof(int) * m->W * m->W,
                               cudaMemcpyHostToDevice, st));
  OAM_CUDA_TRY(cudaMallocAsync((void **)&d_orb_b, sizeof(int) * O, st));
  OAM_CUDA_TRY(cudaMallocAsync((void **)&d_orb_a, sizeof(int) * O, st));
  OAM_CUDA_TRY(cudaMallocAsync((void **)&d_range, sizeof(double2) * O * nz, st));
  OAM_CUDA_TRY(cudaMemcpyAsync(d_orb_b, m->h_orb_b.data(), sizeof(int) * O, cudaMemcpyHostToDevice, st));
  OAM_CUDA_TRY(cudaMemcpyAsync(d_orb_a, m->h_orb_a.data(), sizeof(int) * O, cudaMemcpyHostToDevice, st));

  Geo g{};
  g.F = m->sensor.focal_m;
  g.dx = gr.dx_m;
  g.dy = gr.dy_m;
  g.dz = gr.dz_m;
  g.z0 = gr.z0_rel_m;
  g.ks = gr.fs_hz / m->sensor.c_mps;
  g.cut = m->cut;
  g.inv2s2 = (float)(1.0 / (2.0 * m->sigma_s * m->sigma_s));
  g.env2 = (float)(1.0 / (2.0 * m->sigma_s * m->sigma_s * std::log(2.0)));
  g.invs2 = (float)(1.0 / (m->sigma_s * m->sigma_s));
  g.omega = (float)m->omega;
  g.cyc = (float)(m->omega / M_PI);

  PatchDW *d_pdw = nullptr;  // double-word patches, freed with the other temporaries
  OAM_CUDA_TRY(cudaMallocAsync((void **)&d_pdw, sizeof(PatchDW) * m->M, st));
  k_patch_dw<<<(m->M + 255) / 256, 256, 0, st>>>(m->d_patch, m->M, d_pdw);
  OAM_LAUNCHED();
  k_delta_range<<<dim3(O, nz), 256, 0, st>>>(g, m->d_patch, d_pdw, m->M, d_orb_b, d_orb_a, nz, d_range);
  OAM_LAUNCHED();
  std::vector<double2> h_range((size_t)O * nz);
  OAM_CUDA_TRY(cudaMemcpyAsync(h_range.data(), d_range, sizeof(double2) * O * nz, cudaMemcpyDeviceToHost, st));
  OAM_CUDA_TRY(cudaStreamSynchronize(st));

  rc = plan_bands(m, h_range, 0);
  if (rc) {
    cudaFreeAsync(d_orb_b, st);
    cudaFreeAsync(d_orb_a, st);
    cudaFreeAsync(d_range, st);
    cudaFreeAsync(d_pdw, st);
    return rc;
  }
  g.G = m->G;

  int *d_band_hi = nullptr;
  if ((rc = dev_alloc(m, &m->d_band_lo, (size_t)O * nz))) return rc;
  OAM_CUDA_TRY(cudaMallocAsync((void **)&d_band_hi, sizeof(int) * O * nz, st));
  OAM_CUDA_TRY(cudaMemcpyAsync(m->d_band_lo, m->h_band_lo.data(), sizeof(int) * O * nz, cudaMemcpyHostToDevice, st));
  OAM_CUDA_TRY(cudaMemcpyAsync(d_band_hi, m->h_band_hi.data(), sizeof(int) * O * nz, cudaMemcpyHostToDevice, st));
  if ((rc = dev_alloc(m, &m->d_band, (size_t)O * nz * m->band_w))) return rc;
  if (m->disc == OAM_DISC_TRILINEAR) {
    Geo33 g3{};
    g3.F = m->sensor.focal_m * 1e3;
    g3.dx = gr.dx_m * 1e3;
    g3.dy = gr.dy_m * 1e3;
    g3.dz = gr.dz_m * 1e3;
    g3.z0 = gr.z0_rel_m * 1e3;
    g3.c = m->sensor.c_mps * 1e3;
    g3.fs = gr.fs_hz;
    g3.t0 = m->t0;
    g3.sigma = m->sigma_s;
    g3.omega = m->omega;
    g3.T = (int)std::floor(m->cut);
    g3.len = (int)std::ceil(2.0 * gr.fs_hz * (gr.dx_m + gr.dy_m + gr.dz_m) / m->sensor.c_mps) + 4;
    const int threads = std::max(128, ((m->band_w + 3) / 4 + 31) & ~31);
    const size_t sm = sizeof(double) * (2 * g3.T + 1 + (size_t)k33Chunk * g3.len) + sizeof(int) * (k33Chunk + 2) +
                      sizeof(double) * k33Chunk;
    if (threads > 1024 || sm > 200 * 1024) return OAM_ERR_UNSUPPORTED;
    if (sm > 48 * 1024) OAM_CUDA_TRY(cudaFuncSetAttribute(k_slab33_values, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_slab33_values<<<dim3(O, nz), threads, sm, st>>>(g3, m->d_patch, m->M, d_orb_b, d_orb_a, nz, nt, m->d_band_lo,
                                                      d_band_hi, m->band_w, m->d_band);
  } else {
    const int threads = m->band_w <= 128 ? 128 : 256;
    const int T0 = (int)std::floor(m->cut + 0.5) + 1;  // rotation table half-length
    k_slab_values<<<dim3(O, nz), threads, sizeof(float2) * (2 * T0 + 1), st>>>(
        g, d_pdw, m->M, d_orb_b, d_orb_a, nz, m->d_band_lo, d_band_hi, m->band_w, T0, m->d_band);
  }
  OAM_LAUNCHED();

  // FP32 forward layout
  m->n_ttiles = (nt + kTimeTile - 1) / kTimeTile;
  {
    const int NT = m->n_ttiles;
    std::vector<int> kr;
    std::vector<long long> off;
    const long long total = fwd_layout(m, &kr, &off);
    if ((rc = dev_alloc(m, &m->d_fwd_krange, kr.size()))) return rc;
    if ((rc = dev_alloc(m, &m->d_fwd_off, off.size()))) return rc;
    if ((rc = dev_alloc(m, &m->d_fwd, (size_t)total))) return rc;
    OAM_CUDA_TRY(cudaMemcpyAsync(m->d_fwd_krange, kr.data(), sizeof(int) * kr.size(), cudaMemcpyHostToDevice, st));
    OAM_CUDA_TRY(cudaMemcpyAsync(m->d_fwd_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, st));
    k_pack_fwd<<<O * NT, 256, 0, st>>>(m->d_band, m->d_band_lo, d_band_hi, m->band_w, nz, NT, m->d_fwd_krange,
                                       m->d_fwd_off, m->d_fwd);
    OAM_LAUNCHED();
    OAM_CUDA_TRY(cudaStreamSynchronize(st));  // host tables above go out of scope
  }
  // FP32 adjoint layout
  m->n_ktiles = (nz + kDepthTile - 1) / kDepthTile;
  {
    const int NK = m->n_ktiles;
    std::vector<int> nr;
    std::vector<long long> off;
    const long long total = adj_layout(m, &nr, &off);
    if ((rc = dev_alloc(m, &m->d_adj_nrange, nr.size()))) return rc;
    if ((rc = dev_alloc(m, &m->d_adj_off, off.size()))) return rc;
    if ((rc = dev_alloc(m, &m->d_adj, (size_t)total))) return rc;
    OAM_CUDA_TRY(cudaMemcpyAsync(m->d_adj_nrange, nr.data(), sizeof(int) * nr.size(), cudaMemcpyHostToDevice, st));
    OAM_CUDA_TRY(cudaMemcpyAsync(m->d_adj_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, st));
    k_pack_adj<<<O * NK, 256, 0, st>>>(m->d_band, m->d_band_lo, d_band_hi, m->band_w, nz, NK, m->d_adj_nrange,
                                       m->d_adj_off, m->d_adj);
    OAM_LAUNCHED();
    OAM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(d_orb_b, st);
  cudaFreeAsync(d_orb_a, st);
  cudaFreeAsync(d_range, st);
  cudaFreeAsync(d_pdw, st);
  cudaFreeAsync(d_band_hi, st);
  return OAM_OK;
}

oam_status oam::slab_column(const oam_model *m, int b, int a, int k, float *d_out, cudaStream_t st) {
  const int o = m->h_tap_orbit[(b + m->R) * m->W + (a + m->R)];
  k_slab_column<<<(m->grid.nt + 255) / 256, 256, 0, st>>>(m->d_band, m->d_band_lo, m->band_w, m->grid.nz,
                                                          m->grid.nt, o, k, d_out);
  OAM_LAUNCHED();
  return OAM_OK;
}
