// Internal declarations shared by the translation units of liboam.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <utility>
#include <vector>

#include "../../include/oam.h"

namespace oam {

constexpr int kTimeTile = 64;  // FP32 forward layout: samples per time tile
constexpr int kDepthTile = 16; // FP32 adjoint layout: depths per depth tile
constexpr int kRedBlocks = 1024; // max blocks of a reduction kernel (partials buffer size)

// Sensor ring plan (host): rings uniform in polar angle, 8*u_r patches each.
struct Ring {
  double cos_mid;  // cosine of the ring's mid polar angle (mean of edge cosines)
  double area;     // ring area, m^2
  int32_t count;   // patches in the ring (multiple of 8)
  int32_t first;   // index of the ring's first patch
};

// One sensor patch (Eq. 3): unit normal n (surface point -F n about the focus)
// and area in mm^2.
struct __align__(32) Patch {
  double x, y, z, w;
};

// Tensor-core operator layout of one direction (forward or adjoint); defined in op_tc.cu.
struct TcLayout;
// Lateral-FFT form of the operators (OAM_PREC_FFT); defined in op_fft.cu.
struct FftLayout;
// Band-pass filter along time of a filtered model; defined in op_filter.cu.
struct FirLayout;

}  // namespace oam

// The opaque model.  All d_* members are device memory owned by the model.
struct oam_model {
  oam_sensor sensor;
  oam_grid grid;
  oam_eir eir;
  int precision;
  int disc = OAM_DISC_POINT;  // oam_discretisation of Eq. 1
  int R, W;                 // half window, window (taps per lateral axis)
  double t0;                // time of sample 0 (s)
  double sigma_s, omega, cut; // EIR in sample units: std dev, angular freq, truncation
  double G;                 // fs * (F/c - t0): sample index of a focal arrival
  int n_lo, n_hi;           // union of all bands
  int n_orb;                // orbits (distinct |offsets| up to x<->y swap when dx == dy)
  std::vector<int> h_tap_orbit;   // [W*W]
  std::vector<int> h_orb_b, h_orb_a;  // representative tap of each orbit
  int *d_tap_orbit = nullptr;

  int M = 0;
  oam::Patch *d_patch = nullptr;  // sensor patches

  // band form of the slab: per (orbit, depth) a band [lo, hi) of samples
  int band_w = 0;                 // stored width (multiple of 4)
  std::vector<int> h_band_lo, h_band_hi;  // [n_orb*nz]
  int *d_band_lo = nullptr;
  float *d_band = nullptr;        // [n_orb][nz][band_w]

  // FP32 forward layout: per (orbit, time tile) depths [klo, khi), rows of kTimeTile samples
  int n_ttiles = 0;
  int *d_fwd_krange = nullptr;    // [n_orb*n_ttiles][2]
  long long *d_fwd_off = nullptr; // [n_orb*n_ttiles]
  float *d_fwd = nullptr;
  // FP32 adjoint layout: per (orbit, depth tile) samples [nlo, nlo+nlen), rows of nlen
  int n_ktiles = 0;
  int *d_adj_nrange = nullptr;    // [n_orb*n_ktiles][2] = (nlo, nlen)
  long long *d_adj_off = nullptr;
  float *d_adj = nullptr;

  // tensor-core layouts (OAM_PREC_BF16X3) and the staging buffer for the
  // split-BF16 copy of the operator input ([chunks][qtot][8] hi, then lo)
  oam::TcLayout *tc_fwd = nullptr;
  oam::TcLayout *tc_adj = nullptr;
  uint8_t *d_tc_pack = nullptr;
  size_t tc_pack_bytes = 0;
  long long tc_qtot = 0;
  float *d_tc_part = nullptr;  // per-part partial sums of the tensor-core operators

  oam::FftLayout *fft = nullptr;  // lateral-FFT form (OAM_PREC_FFT)
  oam::FirLayout *fir = nullptr;  // band-pass filter: forward is F A, adjoint A^T F (none: nullptr)
  unsigned generation = 0;        // bumped when the operators' buffers change (filter set or removed)

  int *d_status = nullptr;  // device error word (bounded waits that ran out)
  cudaStream_t alloc_stream = nullptr;  // stream of the stream-ordered allocations (the build stream)

  // operator timing (oam_profile_enable / oam_profile_read)
  struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<std::pair<size_t, size_t>> fwd, adj;
  };
  mutable Prof prof;

  long long nnz = 0;
  double flops = 0;
  size_t bytes = 0;
  int sm_count = 0;
};

namespace oam {

// ---- helpers --------------------------------------------------------------
extern std::atomic<long long> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Event pair around one operator kernel when profiling is on (else no-op).
struct ProfScope {
  const oam_model *m;
  cudaStream_t st;
  bool fwd;
  size_t first = 0;
  bool active = false;
  ProfScope(const oam_model *m_, cudaStream_t s, bool f);
  ~ProfScope();
};

#define OAM_CUDA_TRY(expr)                        \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return OAM_ERR_CUDA;   \
  } while (0)

// After every kernel launch: count it and surface launch errors.
#define OAM_LAUNCHED()                                  \
  do {                                                  \
    ::oam::count_launch();                              \
    OAM_CUDA_TRY(cudaGetLastError());                   \
  } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Bytes dev_alloc reserves for `count` elements of T (an empty array still takes one).
template <typename T>
inline size_t alloc_bytes(size_t count) {
  return (count ? count : 1) * sizeof(T);
}

// slab.cu
oam_status build_slab(oam_model *m, cudaStream_t st);
oam_status plan_bands(oam_model *m, const std::vector<double2> &h_range, int widen);
long long fwd_layout(const oam_model *m, std::vector<int> *kr, std::vector<long long> *off);
long long adj_layout(const oam_model *m, std::vector<int> *nr, std::vector<long long> *off);
size_t slab_plan_bytes(const oam_model *m);
oam_status slab_column(const oam_model *m, int b, int a, int k, float *d_out, cudaStream_t st);

// op_fp32.cu
oam_status forward_fp32(const oam_model *m, const float *H, float *s, cudaStream_t st);
oam_status adjoint_fp32(const oam_model *m, const float *s, float *H, cudaStream_t st);

// op_tc.cu
oam_status tc_build(oam_model *m, cudaStream_t st);
void tc_free(oam_model *m, cudaStream_t st);
oam_status forward_tc(const oam_model *m, const float *H, float *s, cudaStream_t st);
oam_status adjoint_tc(const oam_model *m, const float *s, float *H, cudaStream_t st);
double tc_exec_flops(const oam_model *m, int dir);
oam_status tc_plan_bytes(const oam_model *m, size_t *bytes);
oam_status tc_autotune(oam_model *m, int reps, cudaStream_t st, int *best_fwd, int *best_adj, int *warps_fwd,
                       int *warps_adj);
oam_status tc_set_tiles(oam_model *m, int dir, int fold_warps, int ring);
void tc_get_tiles(const oam_model *m, int dir, int *fold_warps, int *ring);
// Position tiling of the split-BF16 kernels (0 auto, 1 padded grid, 2 scan grid).
oam_status tc_set_tiling(oam_model *m, int dir, int tiling);
int tc_get_tiling(const oam_model *m, int dir);

// op_fft.cu
oam_status fft_build(oam_model *m, cudaStream_t st);
void fft_free(oam_model *m, cudaStream_t st);
oam_status forward_fft(const oam_model *m, const float *H, float *s, cudaStream_t st);
oam_status adjoint_fft(const oam_model *m, const float *s, float *H, cudaStream_t st);
double fft_flops(const oam_model *m);
double fft_bytes(const oam_model *m);
oam_status fft_plan_bytes(const oam_model *m, size_t *bytes);

// op_filter.cu: y = F x over the model's py*px A-lines (x and y may alias)
oam_status fir_apply(const oam_model *m, const float *x, float *y, cudaStream_t st);
float *fir_stage(const oam_model *m);
int fir_half_len(const oam_model *m);
int fir_size(const oam_model *m);
void fir_free(oam_model *m, cudaStream_t st);

// samples by which a trilinear voxel's arrivals (and the finite difference)
// extend the point voxel's: ceil(fs (dx + dy + dz) / c) + 2; 0 for point voxels
int disc_margin(const oam_model *m);

// free every device buffer of a model with cudaFreeAsync on `st`, then the model
void model_release(oam_model *m, cudaStream_t st);

// dispatch on the model's precision
oam_status apply_forward(const oam_model *m, const float *H, float *s, cudaStream_t st);
oam_status apply_adjoint(const oam_model *m, const float *s, float *H, cudaStream_t st);

inline size_t vol_elems(const oam_model *m) {
  return (size_t)m->grid.py * m->grid.px * m->grid.nz;
}
inline size_t sig_elems(const oam_model *m) {
  return (size_t)m->grid.py * m->grid.px * m->grid.nt;
}

// Model memory comes from the stream-ordered allocator on the build stream, so
// releasing a model never forces a device-wide synchronisation.
template <typename T>
oam_status dev_alloc(oam_model *m, T **p, size_t count) {
  if (count == 0) count = 1;
  if (cudaMallocAsync((void **)p, count * sizeof(T), m->alloc_stream) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return OAM_ERR_OOM;
  }
  m->bytes += count * sizeof(T);
  return OAM_OK;
}

}  // namespace oam
