// Plain FP32 forward and adjoint operators on CUDA cores.
//
// Both are lateral correlations of the single-position slab with the volume or
// the signals ("two coordinate systems": the absolute index of a voxel and its
// offset relative to each scan position; Methods, Efficient reconstruction
// based on scanning symmetries).  Voxels and samples outside the grids are zero.
//
// forward: block = (row y, 64 positions, 64-sample time tile); it walks every
//   tap (b, a) and the depths whose band meets the time tile, staging 16 depths
//   of the shifted volume row and the packed slab rows in shared memory.
// adjoint: block = (row y, 64 positions, 16-depth tile), 64 threads of 4
//   positions x 4 depths; it walks every tap and the samples of the tile's band
//   union, 64 samples at a time.
//
// Each output sums up to win^2 x band products (about 3e5 at 61 x 61 taps).
// One FP32 accumulator for all of them loses about sqrt(n) units in the last
// place, 2e-5 relative at that size, so both kernels sum in three levels: the
// products of one tap, then the taps of one tap row, then the rows.
#include "internal.cuh"

using namespace oam;

namespace {

constexpr int kPos = 64;

__global__ void __launch_bounds__(256) k_fwd_fp32(const float *__restrict__ H, float *__restrict__ s, int px, int py,
                                                  int nz, int nt, int R, const int *__restrict__ tap_orbit, int n_tt,
                                                  const int *__restrict__ krange, const long long *__restrict__ off,
                                                  const float *__restrict__ P) {
  const int x0 = blockIdx.x * kPos, y = blockIdx.y, T = blockIdx.z;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int W = 2 * R + 1;
  __shared__ __align__(16) float Hs[kPos][kDepthTile + 4];  // rows of 16 depths, 16-byte aligned
  __shared__ float4 Ps[kDepthTile][kTimeTile / 4];
  float acc[4][4] = {}, row_acc[4][4], tap_acc[4][4];
  for (int b = -R; b <= R; ++b) {
    const int yy = y + b;
    if (yy < 0 || yy >= py) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) row_acc[i][j] = 0.0f;
    for (int a = -R; a <= R; ++a) {
      const int xs = x0 + a;
      if (xs + kPos <= 0 || xs >= px) continue;
      const int oi = tap_orbit[(b + R) * W + (a + R)] * n_tt + T;
      const int klo = krange[2 * oi], khi = krange[2 * oi + 1];
      if (klo >= khi) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) tap_acc[i][j] = 0.0f;
      const float4 *P4 = reinterpret_cast<const float4 *>(P + off[oi]);
      // this thread's share of a 16-depth chunk (4 volume values, 4 slab values),
      // fetched one chunk ahead so the loads run during the previous chunk's FMAs
      float hv[4];
      float4 pv;
      auto fetch = [&](int kc) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int e = tid + 256 * r, p = e >> 4, kk = e & 15;
          const int x = xs + p, k = kc + kk;
          hv[r] = (x >= 0 && x < px && k < khi) ? H[((size_t)yy * px + x) * nz + k] : 0.0f;
        }
        const int row = tid >> 4, c4 = tid & 15;
        pv = (kc + row < khi) ? P4[(size_t)(kc - klo + row) * (kTimeTile / 4) + c4] : make_float4(0.f, 0.f, 0.f, 0.f);
      };
      fetch(klo);
      for (int kc = klo; kc < khi; kc += kDepthTile) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int e = tid + 256 * r;
          Hs[e >> 4][e & 15] = hv[r];
        }
        Ps[tid >> 4][tid & 15] = pv;
        __syncthreads();
        if (kc + kDepthTile < khi) fetch(kc + kDepthTile);
        // four depths per step: 4 + 4 16-byte reads for 64 FMAs, each
        // accumulator still taking its depths in increasing order
#pragma unroll
        for (int k4 = 0; k4 < kDepthTile; k4 += 4) {
          float4 p[4], h[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) p[u] = Ps[k4 + u][tx];
#pragma unroll
          for (int i = 0; i < 4; ++i) h[i] = *reinterpret_cast<const float4 *>(&Hs[4 * ty + i][k4]);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float hv = u == 0 ? h[i].x : u == 1 ? h[i].y : u == 2 ? h[i].z : h[i].w;
              tap_acc[i][0] = fmaf(hv, p[u].x, tap_acc[i][0]);
              tap_acc[i][1] = fmaf(hv, p[u].y, tap_acc[i][1]);
              tap_acc[i][2] = fmaf(hv, p[u].z, tap_acc[i][2]);
              tap_acc[i][3] = fmaf(hv, p[u].w, tap_acc[i][3]);
            }
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) row_acc[i][j] += tap_acc[i][j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += row_acc[i][j];
  }
  const int n = T * kTimeTile + 4 * tx;
  if (n >= nt) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int x = x0 + 4 * ty + i;
    if (x < px)
      *reinterpret_cast<float4 *>(s + ((size_t)y * px + x) * nt + n) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

constexpr int kAdjThreads = 64;

__global__ void __launch_bounds__(kAdjThreads) k_adj_fp32(const float *__restrict__ s, float *__restrict__ H, int px,
                                                          int py, int nz, int nt, int R,
                                                          const int *__restrict__ tap_orbit, int n_kt,
                                                          const int *__restrict__ nrange,
                                                          const long long *__restrict__ off,
                                                          const float *__restrict__ Q) {
  const int x0 = blockIdx.x * kPos, y = blockIdx.y, K = blockIdx.z;
  // thread: positions pg + 16 i (i < 4) and depths 4 dg + d (d < 4) of the tile
  const int tid = threadIdx.x, pg = tid & 15, dg = tid >> 4;
  const int W = 2 * R + 1;
  __shared__ float4 Ss[kPos][kTimeTile / 4 + 1];
  __shared__ float4 Qs[kDepthTile][kTimeTile / 4];
  float acc[4][4] = {}, row_acc[4][4], tap_acc[4][4];
  for (int b = -R; b <= R; ++b) {
    const int yy = y - b;
    if (yy < 0 || yy >= py) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int d = 0; d < 4; ++d) row_acc[i][d] = 0.0f;
    for (int a = -R; a <= R; ++a) {
      const int xs = x0 - a;
      if (xs + kPos <= 0 || xs >= px) continue;
      const int oi = tap_orbit[(b + R) * W + (a + R)] * n_kt + K;
      const int nlo = nrange[2 * oi], nlen = nrange[2 * oi + 1];
      if (nlen <= 0) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int d = 0; d < 4; ++d) tap_acc[i][d] = 0.0f;
      const float4 *Q4 = reinterpret_cast<const float4 *>(Q + off[oi]);
      for (int nc = 0; nc < nlen; nc += kTimeTile) {
#pragma unroll 4
        for (int r = 0; r < kPos * (kTimeTile / 4) / kAdjThreads; ++r) {
          const int e = tid + kAdjThreads * r, pp = e >> 4, j4 = e & 15;
          const int x = xs + pp, j = nc + 4 * j4;
          Ss[pp][j4] = (x >= 0 && x < px && j < nlen)
                           ? *reinterpret_cast<const float4 *>(s + ((size_t)yy * px + x) * nt + nlo + j)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < kDepthTile * (kTimeTile / 4) / kAdjThreads; ++r) {
          const int e = tid + kAdjThreads * r, row = e >> 4, j4 = e & 15, j = nc + 4 * j4;
          Qs[row][j4] = (j < nlen) ? Q4[((size_t)row * nlen + j) >> 2] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        // 4 + 4 16-byte reads for 64 FMAs; each accumulator takes its samples
        // in increasing order
#pragma unroll 2
        for (int j4 = 0; j4 < kTimeTile / 4; ++j4) {
          float4 v[4], q[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) v[i] = Ss[pg + 16 * i][j4];
#pragma unroll
          for (int d = 0; d < 4; ++d) q[d] = Qs[4 * dg + d][j4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int d = 0; d < 4; ++d) {
              tap_acc[i][d] = fmaf(v[i].x, q[d].x, tap_acc[i][d]);
              tap_acc[i][d] = fmaf(v[i].y, q[d].y, tap_acc[i][d]);
              tap_acc[i][d] = fmaf(v[i].z, q[d].z, tap_acc[i][d]);
              tap_acc[i][d] = fmaf(v[i].w, q[d].w, tap_acc[i][d]);
            }
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int d = 0; d < 4; ++d) row_acc[i][d] += tap_acc[i][d];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int d = 0; d < 4; ++d) acc[i][d] += row_acc[i][d];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int x = x0 + pg + 16 * i;
    if (x >= px) continue;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int k = K * kDepthTile + 4 * dg + d;
      if (k < nz) H[((size_t)y * px + x) * nz + k] = acc[i][d];
    }
  }
}

}  // namespace

oam_status oam::forward_fp32(const oam_model *m, const float *H, float *s, cudaStream_t st) {
  const oam_grid &g = m->grid;
  dim3 grid((g.px + kPos - 1) / kPos, g.py, m->n_ttiles);
  ProfScope prof(m, st, true);
  k_fwd_fp32<<<grid, 256, 0, st>>>(H, s, g.px, g.py, g.nz, g.nt, m->R, m->d_tap_orbit, m->n_ttiles, m->d_fwd_krange,
                                   m->d_fwd_off, m->d_fwd);
  OAM_LAUNCHED();
  return OAM_OK;
}

oam_status oam::adjoint_fp32(const oam_model *m, const float *s, float *H, cudaStream_t st) {
  const oam_grid &g = m->grid;
  dim3 grid((g.px + kPos - 1) / kPos, g.py, m->n_ktiles);
  ProfScope prof(m, st, false);
  k_adj_fp32<<<grid, kAdjThreads, 0, st>>>(s, H, g.px, g.py, g.nz, g.nt, m->R, m->d_tap_orbit, m->n_ktiles,
                                           m->d_adj_nrange, m->d_adj_off, m->d_adj);
  OAM_LAUNCHED();
  return OAM_OK;
}
