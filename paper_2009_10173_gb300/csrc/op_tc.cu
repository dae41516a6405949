// Split-BF16 forward and adjoint operators on the 5th-generation tensor cores
// (tcgen05 MMA, accumulators in tensor memory, operands staged by the TMA
// engine).  Both are the lateral correlations of Eq. 4 ("two coordinate
// systems", Methods, Efficient reconstruction based on scanning symmetries)
// written as one implicit GEMM per block of 128 scan positions:
//
//   forward  D[pos][n] += sum_{tap, k}  X[pos + tap][k] * S_tap[k][n]
//   adjoint  D[pos][k] += sum_{tap, n}  X[pos - tap][n] * S_tap[k][n]
//
// M = 128 positions (one tensor-memory lane each), N = the slab band of one
// 16-deep K chunk (time samples for A, depths for A^T), K = (tap, 16-chunk).
// Positions use a padded flat index q = y*Wp + x with Wp = px + R, so a
// lateral tap shift a is a shift of the whole 128-row operand by a rows: one
// staged strip of 128 + 2R rows serves all 2R+1 taps of a row offset b by
// moving the shared-memory descriptor start 16 bytes per tap.  Padding
// columns hold zeros, and out-of-grid rows sit in zero padding rows.
//
// Each product uses hi = bf16(v), lo = bf16(v - hi) splits of the slab and of
// the iterate: D += X_hi S_hi + X_hi S_lo + X_lo S_hi, accumulated in FP32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "internal.cuh"
#include "tc_ptx.cuh"

using namespace oam;

namespace oam {

constexpr int kStageK = 32;        // K elements per staged strip (two 16-deep MMA chunks)
constexpr int kTileM = 128;        // positions per block
constexpr int kThreads = 192;      // warp 0 producer, warp 1 MMA, warps 2-5 epilogue
constexpr int kSmemLimit = 227 * 1024;

struct __align__(16) TcItem {
  uint32_t off16;    // byte offset of the item's tiles in data, in 16-byte units
  uint32_t bytes;    // total bytes (hi + lo of both tiles)
  uint16_t col[2];   // accumulator column of each tile
  uint16_t n[2];     // MMA N of each tile (0 = no tile)
};

struct TcTile {
  int orbit, chunk, col, n;
  long long off;  // byte offset of the hi part; lo follows after n*32 bytes
};

struct TcLayout {
  int dir = 0;            // 0 forward, 1 adjoint
  int stages = 0;         // K stages of kStageK
  int acc_cols = 0;       // accumulator width (multiple of 16)
  int tmem_cols = 0;      // allocated tensor-memory columns (power of two >= 32)
  int out_lo = 0;         // output index of accumulator column 0
  int in_lo = 0;          // input index of packed chunk 0
  int chunks8 = 0;        // 8-element chunks in the packed input
  int slot_bytes = 0;     // shared-memory slot per item
  TcItem *d_items = nullptr;
  uint8_t *d_data = nullptr;
  size_t data_bytes = 0;
  double exec_flops = 0;  // MMA flops of one application (3 products, band and tile padding)
};

}  // namespace oam

namespace {

struct CorrParams {
  const uint8_t *in_hi, *in_lo;  // packed input [chunks8][qtot][8 x bf16]
  long long qtot;
  int wp, px, py, R, W, dir, stages;
  const int *tap_orbit;
  const TcItem *items;  // [n_orb][stages]
  const uint8_t *data;
  int slot_bytes, n_slots, strip_rows, items_bytes;
  int acc_cols, tmem_cols;
  float *part;            // partial sums [W][py*px][acc_cols], one slice per tap row b
  size_t part_stride;     // py*px
  int *status;
  long long budget;
};

__device__ __forceinline__ bool row_skipped(const CorrParams &p, int tile, int b) {
  const int q0 = tile * kTileM;
  const int y_first = q0 / p.wp, y_last = (q0 + kTileM - 1) / p.wp;
  const int off = p.dir == 0 ? b : -b;
  return (y_last + off < 0) || (y_first + off >= p.py);
}

__global__ void __launch_bounds__(kThreads, 1) k_corr_tc(const CorrParams p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  uint64_t *strip_full = bars, *strip_empty = bars + 2;
  uint64_t *acc_ready = bars + 4, *acc_full = bars + 5;
  uint64_t *slab_full = bars + 6, *slab_empty = bars + 6 + p.n_slots;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 256);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 260);
  volatile int *never = reinterpret_cast<volatile int *>(smem + 264);  // stays 0: waits that ignore abort
  const int L = p.strip_rows;
  const uint32_t strip_bytes = (uint32_t)L * 16u * 4u * 2u;  // 4 chunks of 8, hi + lo
  TcItem *sitems = reinterpret_cast<TcItem *>(smem + 512);  // [stages][W] for this block's row
  uint8_t *strips = smem + 512 + p.items_bytes;
  uint8_t *slots = strips + 2 * strip_bytes;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x;
  const int b = (int)blockIdx.y - p.R;  // this block's tap row
  const bool skip_row = row_skipped(p, tile, b);

  if (threadIdx.x == 0) {
    ptx::mbar_init(&strip_full[0], 1);
    ptx::mbar_init(&strip_full[1], 1);
    ptx::mbar_init(&strip_empty[0], 1);
    ptx::mbar_init(&strip_empty[1], 1);
    ptx::mbar_init(acc_ready, 4);
    ptx::mbar_init(acc_full, 1);
    for (int i = 0; i < p.n_slots; ++i) {
      ptx::mbar_init(&slab_full[i], 1);
      ptx::mbar_init(&slab_empty[i], 1);
    }
    *abort_flag = 0;
    *never = 0;
    ptx::mbar_fence_init();
  }
  if (warp == 0 && !skip_row) {
    const int n = p.stages * p.W;
    for (int i = lane; i < n; i += 32) {
      const int st = i / p.W, ai = i % p.W;
      sitems[i] = p.items[p.tap_orbit[(b + p.R) * p.W + ai] * p.stages + st];
    }
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, p.tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto fail = [&](int code) {
    *abort_flag = 1;
    atomicOr(p.status, code);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int it_strip = 0, it_slab = 0;
      bool ok = true;
      if (!skip_row) {
        const long long q_base =
            (long long)(p.R + 1) * p.wp + (long long)tile * kTileM + (long long)(p.dir == 0 ? b : -b) * p.wp - p.R;
        for (int st = 0; st < p.stages && ok; ++st) {
          const int s = it_strip & 1;
          if (!ptx::mbar_wait(&strip_empty[s], ((it_strip >> 1) & 1) ^ 1, abort_flag, p.budget)) {
            fail(1);
            ok = false;
            break;
          }
          ptx::mbar_arrive_expect_tx(&strip_full[s], strip_bytes);
          uint8_t *dst = strips + s * strip_bytes;
          for (int c = 0; c < 4; ++c) {
            const long long src = ((long long)(4 * st + c) * p.qtot + q_base) * 16;
            ptx::bulk_g2s(dst + c * L * 16, p.in_hi + src, L * 16, &strip_full[s]);
            ptx::bulk_g2s(dst + (4 + c) * L * 16, p.in_lo + src, L * 16, &strip_full[s]);
          }
          ++it_strip;
          const TcItem *row_items = sitems + st * p.W;
          for (int ai = 0; ai < p.W; ++ai) {
            const TcItem item = row_items[ai];
            const int slot = it_slab % p.n_slots;
            if (!ptx::mbar_wait(&slab_empty[slot], ((it_slab / p.n_slots) & 1) ^ 1, abort_flag, p.budget)) {
              fail(2);
              ok = false;
              break;
            }
            ptx::mbar_arrive_expect_tx(&slab_full[slot], item.bytes);
            if (item.bytes > 0)
              ptx::bulk_g2s(slots + (size_t)slot * p.slot_bytes, p.data + (size_t)item.off16 * 16, item.bytes,
                            &slab_full[slot]);
            ++it_slab;
          }
        }
      }
      if (!ok) {
        // let copies already issued land before the block exits
        for (int i = std::max(0, it_slab - p.n_slots); i < it_slab; ++i)
          ptx::mbar_wait(&slab_full[i % p.n_slots], (i / p.n_slots) & 1, never, p.budget);
        for (int i = std::max(0, it_strip - 2); i < it_strip; ++i)
          ptx::mbar_wait(&strip_full[i & 1], (i >> 1) & 1, never, p.budget);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool ok = ptx::mbar_wait(acc_ready, 0, abort_flag, p.budget);
      if (!ok) fail(4);
      ptx::tc_fence_after();
      int it_strip = 0, it_slab = 0;
      const uint32_t lbo_a = (uint32_t)L * 16u;
      if (!skip_row) {
        for (int st = 0; st < p.stages && ok; ++st) {
          const int s = it_strip & 1;
          if (!ptx::mbar_wait(&strip_full[s], (it_strip >> 1) & 1, abort_flag, p.budget)) {
            fail(8);
            ok = false;
            break;
          }
          const uint32_t a_hi = ptx::smem_addr(strips + s * strip_bytes);
          const uint32_t a_lo = a_hi + 4u * lbo_a;
          const TcItem *row_items = sitems + st * p.W;
          for (int ai = 0; ai < p.W; ++ai) {
            const TcItem item = row_items[ai];
            const int slot = it_slab % p.n_slots;
            if (!ptx::mbar_wait(&slab_full[slot], (it_slab / p.n_slots) & 1, abort_flag, p.budget)) {
              fail(16);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            // tap a = ai - R: forward reads row m + R + a, adjoint row m + R - a
            const uint32_t shift = (uint32_t)(p.dir == 0 ? ai : 2 * p.R - ai) * 16u;
            uint32_t b_addr = ptx::smem_addr(slots + (size_t)slot * p.slot_bytes);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              const uint32_t N = item.n[c];
              if (N == 0) continue;
              const uint32_t idesc = ptx::idesc_bf16_f32(kTileM, N);
              const uint64_t dah = ptx::smem_desc(a_hi + 2u * c * lbo_a + shift, lbo_a, 128);
              const uint64_t dal = ptx::smem_desc(a_lo + 2u * c * lbo_a + shift, lbo_a, 128);
              const uint64_t dbh = ptx::smem_desc(b_addr, N * 16u, 128);
              const uint64_t dbl = ptx::smem_desc(b_addr + N * 32u, N * 16u, 128);
              const uint32_t d = tmem + item.col[c];
              ptx::mma_bf16(d, dah, dbh, idesc, 1);
              ptx::mma_bf16(d, dah, dbl, idesc, 1);
              ptx::mma_bf16(d, dal, dbh, idesc, 1);
              b_addr += N * 64u;
            }
            ptx::mma_commit(&slab_empty[slot]);
            ++it_slab;
          }
          ptx::mma_commit(&strip_empty[s]);
          ++it_strip;
        }
      }
      ptx::mma_commit(acc_full);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2-5)
    const int quarter = warp & 3;  // tensor-memory lanes 32*quarter .. +31
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    for (int col = 0; col < p.tmem_cols; col += 32) ptx::tmem_st32_zero(tmem + lane_base + (uint32_t)col);
    ptx::tmem_wait_st();
    ptx::tc_fence_before();
    __syncwarp();
    if (lane == 0) ptx::mbar_arrive(acc_ready);
    bool ok = ptx::mbar_wait(acc_full, 0, abort_flag, 4 * p.budget);
    ok = __all_sync(0xffffffffu, ok);
    ptx::tc_fence_after();
    const int m = 32 * quarter + lane;
    const long long qf = (long long)tile * kTileM + m;
    const int y = (int)(qf / p.wp), x = (int)(qf % p.wp);
    const bool valid = ok && y < p.py && x < p.px;
    // this part's partial sums: part[blockIdx.y][y*px + x][0 .. acc_cols)
    float *row = p.part + ((size_t)blockIdx.y * p.part_stride + (size_t)y * p.px + x) * p.acc_cols;
    if (ok) {
      for (int col = 0; col < p.acc_cols; col += 32) {
        uint32_t r[32];
        ptx::tmem_ld32(tmem + lane_base + (uint32_t)col, r);
        ptx::tmem_wait_ld();
        if (valid) {
          float4 *dst = reinterpret_cast<float4 *>(row + col);
          const int nv = min(8, (p.acc_cols - col) >> 2);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j < nv)
              dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                   __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
        }
      }
    }
    ptx::tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, p.tmem_cols);
  }
}

// ---------------------------------------------------------------- packers
// Slab tiles: hi then lo, each [2 chunks of 8][n rows][8] bf16 (K-major core matrices).
__global__ void k_pack_tiles(const float *band, const int *band_lo, const int *band_hi, int band_w, int nz,
                             int dir, int t_lo, const TcTile *tiles, uint8_t *data) {
  const TcTile t = tiles[blockIdx.x];
  __nv_bfloat16 *hi = reinterpret_cast<__nv_bfloat16 *>(data + t.off);
  __nv_bfloat16 *lo = hi + 16 * t.n;
  for (int i = threadIdx.x; i < 16 * t.n; i += blockDim.x) {
    const int kk = i / t.n, row = i % t.n;  // kk: index along K (0..15), row: along N
    int k, n;
    if (dir == 0) {
      k = 16 * t.chunk + kk;
      n = t_lo + t.col + row;
    } else {
      k = t.col + row;
      n = t_lo + 16 * t.chunk + kk;
    }
    float v = 0.0f;
    if (k < nz) {
      const int lo_n = band_lo[t.orbit * nz + k], hi_n = band_hi[t.orbit * nz + k];
      if (n >= lo_n && n < hi_n) v = band[((size_t)t.orbit * nz + k) * band_w + (n - lo_n)];
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    const int idx = ((kk >> 3) * t.n + row) * 8 + (kk & 7);
    hi[idx] = h;
    lo[idx] = l;
  }
}

// Iterate: in[py][px][len] (FP32) -> hi/lo [chunks8][qtot][8] bf16, element j of
// chunk c holding index first + 8c + j of the row of padded position q.
__global__ void k_pack_input(const float *__restrict__ in, int len, int first, int chunks8, long long qtot, int wp,
                             int R, int px, int py, uint4 *__restrict__ out_hi, uint4 *__restrict__ out_lo) {
  const long long total = (long long)chunks8 * qtot;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / qtot);
    const long long q = i % qtot;
    const int y = (int)(q / wp) - (R + 1), x = (int)(q % wp);
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.0f;
    if (y >= 0 && y < py && x < px) {
      const float *src = in + ((size_t)y * px + x) * len;
      const int e0 = first + 8 * c;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (e0 + j < len) v[j] = src[e0 + j];
    }
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      h[j] = __float2bfloat16_rn(v[j]);
      l[j] = __float2bfloat16_rn(v[j] - __bfloat162float(h[j]));
    }
    out_hi[i] = *reinterpret_cast<uint4 *>(h);
    out_lo[i] = *reinterpret_cast<uint4 *>(l);
  }
}

// out[pos][n] = sum over parts (in index order) of part[.][pos][n - out_lo] for n
// in the accumulator range, 0 elsewhere.  Every element of out is written.
__global__ void k_sum_parts(const float *__restrict__ part, int parts, size_t npos, int acc_cols, int out_lo,
                            int out_len, float *__restrict__ out) {
  const size_t total = npos * (size_t)out_len;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t pos = i / out_len;
    const int n = (int)(i % out_len), c = n - out_lo;
    float v = 0.0f;
    if (c >= 0 && c < acc_cols) {
      const float *src = part + pos * acc_cols + c;
      for (int q = 0; q < parts; ++q) v += src[(size_t)q * npos * acc_cols];
    }
    out[i] = v;
  }
}

int pow2_cols(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

// Build one direction's item and tile tables from the band form, then pack.
oam_status build_dir(oam_model *m, TcLayout *L, int dir, cudaStream_t st, int *d_band_hi) {
  const int nz = m->grid.nz, O = m->n_orb;
  const int t_lo = m->n_lo & ~15;
  L->dir = dir;
  if (dir == 0) {
    L->stages = (nz + kStageK - 1) / kStageK;
    L->acc_cols = ((m->n_hi - t_lo) + 15) & ~15;
    L->out_lo = t_lo;
    L->in_lo = 0;
  } else {
    L->stages = ((m->n_hi - t_lo) + kStageK - 1) / kStageK;
    L->acc_cols = (nz + 15) & ~15;
    L->out_lo = 0;
    L->in_lo = t_lo;
  }
  L->chunks8 = 4 * L->stages;
  L->tmem_cols = pow2_cols(L->acc_cols);
  if (L->tmem_cols > 512) return OAM_ERR_UNSUPPORTED;

  std::vector<TcItem> items((size_t)O * L->stages);
  std::vector<TcTile> tiles;
  long long off = 0;
  int max_item = 16;
  double flops_cols = 0;  // sum over orbits of MMA columns x 16 (per position, per tap)
  for (int o = 0; o < O; ++o) {
    for (int s = 0; s < L->stages; ++s) {
      TcItem it{};
      const long long item_off = off;
      if (off / 16 > 0xFFFFFFFFLL) return OAM_ERR_UNSUPPORTED;
      it.off16 = (uint32_t)(off / 16);
      for (int c = 0; c < 2; ++c) {
        const int chunk = 2 * s + c;
        int lo = 1 << 30, hi = -1;
        if (dir == 0) {
          for (int k = 16 * chunk; k < std::min(nz, 16 * chunk + 16); ++k) {
            const int bl = m->h_band_lo[(size_t)o * nz + k], bh = m->h_band_hi[(size_t)o * nz + k];
            if (bh > bl) {
              lo = std::min(lo, bl - t_lo);
              hi = std::max(hi, bh - t_lo);
            }
          }
        } else {
          const int n0 = t_lo + 16 * chunk, n1 = n0 + 16;
          for (int k = 0; k < nz; ++k) {
            const int bl = m->h_band_lo[(size_t)o * nz + k], bh = m->h_band_hi[(size_t)o * nz + k];
            if (bh > bl && bl < n1 && bh > n0) {
              lo = std::min(lo, k);
              hi = std::max(hi, k + 1);
            }
          }
        }
        if (hi <= lo) {
          it.col[c] = 0;
          it.n[c] = 0;
          continue;
        }
        const int col = lo & ~15;
        const int n = ((hi - col) + 15) & ~15;
        if (n > 256 || col + n > L->acc_cols) return OAM_ERR_UNSUPPORTED;
        it.col[c] = (uint16_t)col;
        it.n[c] = (uint16_t)n;
        tiles.push_back(TcTile{o, chunk, col, n, off});
        off += 64LL * n;  // hi + lo: 2 x (n rows x 16 elements x 2 bytes)
        flops_cols += 16.0 * n;
      }
      it.bytes = (uint32_t)(off - item_off);
      max_item = std::max(max_item, (int)it.bytes);
      items[(size_t)o * L->stages + s] = it;
    }
  }
  L->slot_bytes = (max_item + 127) & ~127;
  L->data_bytes = (size_t)std::max<long long>(off, 16);
  // executed MMA flops of one application: 3 products x 2 x M x (16 x N) summed
  // over the (position tile, tap row) blocks whose row meets the grid
  {
    std::vector<double> orb_cols(O, 0.0);
    for (const TcTile &t : tiles) orb_cols[t.orbit] += 16.0 * t.n;
    const int wp = m->grid.px + m->R, W = m->W, R = m->R;
    const long long n_tiles = ((long long)m->grid.py * wp + kTileM - 1) / kTileM;
    std::vector<double> row_cols(W, 0.0);
    for (int bi = 0; bi < W; ++bi)
      for (int ai = 0; ai < W; ++ai) row_cols[bi] += orb_cols[m->h_tap_orbit[bi * W + ai]];
    double total = 0;
    for (long long t = 0; t < n_tiles; ++t) {
      const long long yf = t * kTileM / wp, yl = (t * kTileM + kTileM - 1) / wp;
      for (int bi = 0; bi < W; ++bi) {
        const int off = dir == 0 ? bi - R : R - bi;
        if (yl + off < 0 || yf + off >= m->grid.py) continue;
        total += row_cols[bi];
      }
    }
    L->exec_flops = 3.0 * 2.0 * kTileM * total;
  }
  oam_status rc;
  if ((rc = dev_alloc(m, &L->d_items, items.size()))) return rc;
  if ((rc = dev_alloc(m, &L->d_data, L->data_bytes))) return rc;
  OAM_CUDA_TRY(cudaMemcpyAsync(L->d_items, items.data(), sizeof(TcItem) * items.size(), cudaMemcpyHostToDevice, st));
  if (!tiles.empty()) {
    TcTile *d_tiles = nullptr;
    OAM_CUDA_TRY(cudaMallocAsync((void **)&d_tiles, sizeof(TcTile) * tiles.size(), st));
    OAM_CUDA_TRY(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TcTile) * tiles.size(), cudaMemcpyHostToDevice, st));
    k_pack_tiles<<<(unsigned)tiles.size(), 256, 0, st>>>(m->d_band, m->d_band_lo, d_band_hi, m->band_w, nz, dir,
                                                         t_lo, d_tiles, L->d_data);
    OAM_LAUNCHED();
    OAM_CUDA_TRY(cudaStreamSynchronize(st));
    OAM_CUDA_TRY(cudaFreeAsync(d_tiles, st));
  }
  return OAM_OK;
}

oam_status run_corr(const oam_model *m, const TcLayout *L, const float *in, int in_len, float *out, int out_len,
                    cudaStream_t st) {
  if (!m->d_tc_part) return OAM_ERR_UNSUPPORTED;
  const int R = m->R, wp = m->grid.px + R;
  const long long qtot = m->tc_qtot;
  uint8_t *hi = m->d_tc_pack, *lo = m->d_tc_pack + (size_t)L->chunks8 * qtot * 16;
  {
    const long long total = (long long)L->chunks8 * qtot;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * m->sm_count);
    k_pack_input<<<blocks, 256, 0, st>>>(in, in_len, L->in_lo, L->chunks8, qtot, wp, R, m->grid.px, m->grid.py,
                                         reinterpret_cast<uint4 *>(hi), reinterpret_cast<uint4 *>(lo));
    OAM_LAUNCHED();
  }
  CorrParams p{};
  p.in_hi = hi;
  p.in_lo = lo;
  p.qtot = qtot;
  p.wp = wp;
  p.px = m->grid.px;
  p.py = m->grid.py;
  p.R = R;
  p.W = m->W;
  p.dir = L->dir;
  p.stages = L->stages;
  p.tap_orbit = m->d_tap_orbit;
  p.items = L->d_items;
  p.data = L->d_data;
  p.slot_bytes = L->slot_bytes;
  p.strip_rows = kTileM + 2 * R;
  p.items_bytes = (int)((sizeof(TcItem) * L->stages * m->W + 127) & ~size_t(127));
  const int strip_bytes = p.strip_rows * 16 * 8;
  p.n_slots = std::min(12, (kSmemLimit - 512 - p.items_bytes - 2 * strip_bytes) / L->slot_bytes);
  if (p.n_slots < 2) return OAM_ERR_UNSUPPORTED;
  p.acc_cols = L->acc_cols;
  p.tmem_cols = L->tmem_cols;
  p.part = m->d_tc_part;
  p.part_stride = (size_t)m->grid.py * m->grid.px;
  p.status = m->d_status;
  p.budget = 4000000000LL;  // ~2 s at 2 GHz
  const size_t smem = 512 + (size_t)p.items_bytes + 2 * (size_t)strip_bytes + (size_t)p.n_slots * p.slot_bytes;
  if (smem > (size_t)kSmemLimit) return OAM_ERR_UNSUPPORTED;
  OAM_CUDA_TRY(cudaFuncSetAttribute(k_corr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int n_tiles = (int)(((long long)m->grid.py * wp + kTileM - 1) / kTileM);
  const int parts = m->W;  // one tap row per block
  {
    ProfScope prof(m, st, L->dir == 0);
    k_corr_tc<<<dim3(n_tiles, parts), kThreads, smem, st>>>(p);
    OAM_LAUNCHED();
  }
  const size_t npos = (size_t)m->grid.py * m->grid.px;
  const int blocks = (int)std::min<size_t>((npos * out_len + 255) / 256, 16ull * m->sm_count);
  k_sum_parts<<<blocks, 256, 0, st>>>(m->d_tc_part, parts, npos, L->acc_cols, L->out_lo, out_len, out);
  OAM_LAUNCHED();
  return OAM_OK;
}

}  // namespace

oam_status oam::tc_build(oam_model *m, cudaStream_t st) {
  if (m->grid.px + m->R > (1 << 20)) return OAM_ERR_UNSUPPORTED;
  if (kTileM + 2 * m->R > 1000) return OAM_ERR_UNSUPPORTED;  // strip rows per chunk
  int *d_band_hi = nullptr;
  const size_t nb = (size_t)m->n_orb * m->grid.nz;
  OAM_CUDA_TRY(cudaMallocAsync((void **)&d_band_hi, sizeof(int) * nb, st));
  OAM_CUDA_TRY(cudaMemcpyAsync(d_band_hi, m->h_band_hi.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
  m->tc_fwd = new TcLayout();
  m->tc_adj = new TcLayout();
  oam_status rc = build_dir(m, m->tc_fwd, 0, st, d_band_hi);
  if (!rc) rc = build_dir(m, m->tc_adj, 1, st, d_band_hi);
  cudaFreeAsync(d_band_hi, st);
  if (rc) return rc;
  const int wp = m->grid.px + m->R;
  m->tc_qtot = (long long)(m->grid.py + 2 * m->R + 2) * wp + 256;
  const int chunks = std::max(m->tc_fwd->chunks8, m->tc_adj->chunks8);
  m->tc_pack_bytes = 2ull * chunks * m->tc_qtot * 16;
  rc = dev_alloc(m, &m->d_tc_pack, m->tc_pack_bytes);
  if (rc) return rc;
  // One block per (position tile, tap row): bounds the MMA steps summed into
  // one tensor-memory accumulator; the rows are added in FP32 in a fixed order.
  const int parts = m->W;
  const int acc = std::max(m->tc_fwd->acc_cols, m->tc_adj->acc_cols);
  rc = dev_alloc(m, &m->d_tc_part, (size_t)parts * m->grid.py * m->grid.px * acc);
  if (rc) return rc;
  OAM_CUDA_TRY(cudaMemsetAsync(m->d_tc_pack, 0, m->tc_pack_bytes, st));
  return OAM_OK;
}

void oam::tc_free(oam_model *m) {
  for (TcLayout *L : {m->tc_fwd, m->tc_adj}) {
    if (!L) continue;
    if (L->d_items) cudaFree(L->d_items);
    if (L->d_data) cudaFree(L->d_data);
    delete L;
  }
  m->tc_fwd = m->tc_adj = nullptr;
  if (m->d_tc_pack) cudaFree(m->d_tc_pack);
  m->d_tc_pack = nullptr;
  if (m->d_tc_part) cudaFree(m->d_tc_part);
  m->d_tc_part = nullptr;
}

double oam::tc_exec_flops(const oam_model *m, int dir) {
  const TcLayout *L = dir == 0 ? m->tc_fwd : m->tc_adj;
  return L ? L->exec_flops : 0.0;
}

oam_status oam::forward_tc(const oam_model *m, const float *H, float *s, cudaStream_t st) {
  return run_corr(m, m->tc_fwd, H, m->grid.nz, s, m->grid.nt, st);
}

oam_status oam::adjoint_tc(const oam_model *m, const float *s, float *H, cudaStream_t st) {
  return run_corr(m, m->tc_adj, s, m->grid.nt, H, m->grid.nz, st);
}
