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
//
// Mirror folding.  The sensor is axially symmetric and its patch set is
// mirror-symmetric (Results, axial symmetry), so S[b][a] = S[+-b][+-a] exactly
// (one stored orbit).  The four mirrored taps therefore share one slab tile,
// and their operand rows are summed before the product:
//   F[pos][k] = X[pos + (b, a)] + X[pos + (b, -a)] + X[pos + (-b, a)] + X[pos + (-b, -a)]
// (duplicates dropped when a or b is 0).  One block handles one 128-position
// tile and a group of kBPerBlock consecutive |b|, one after the other into the
// same accumulator; for each it stages the FP32 rows y+b and y-b (TMA, 128-byte
// swizzle) and adds them once per stage, sixteen warps build F from two shifted
// rows of that sum (8 of the stage's 32 K elements each), split it into BF16
// hi/lo in tensor memory, and one warp walks the items while an elected lane
// issues the MMAs with A read from tensor memory.  This cuts the MMA count by
// ~4 for a 61x61 window.
//
// The iterate is packed with a padded flat index q = y*Wp + x, Wp = px + R
// (zero columns px .. Wp-1 and R+1 zero rows above and below), so a lateral
// offset a is a shift by a rows of a staged strip.  A block's 128 positions
// are consecutive in one of two grids (the position tiling, a tile parameter):
// the padded grid (o = y*Wp + x; padding positions compute and are dropped;
// strips of 128 + 2R rows) or the scan grid (o = y*px + x, every lane an
// output; lane m reads strip row m + R*(rows wrapped before m) + R + a, and a
// strip holds 128 + (w + 2) R rows for tiles that wrap w scan rows).
//
// Each product uses hi = bf16(v), lo = bf16(v - hi) splits of the slab and of
// the folded iterate: D += F_hi S_hi + F_hi S_lo + F_lo S_hi, accumulated in
// FP32 in tensor memory.  Each block's tensor-memory sums are written as one
// partial per |b| group; k_sum_parts adds them in index order (this bounds how many
// MMA results any one accumulator takes, which keeps the tensor cores' FP32
// accumulation within 1e-4 of the FP64 oracle).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "internal.cuh"
#include "tc_ptx.cuh"

using namespace oam;

namespace oam {

constexpr int kStageK = 32;        // K elements per stage (two 16-deep MMA chunks)
constexpr int kTileM = 128;        // positions per block
constexpr int kFoldWarpChoices[] = {4, 8, 16};  // warps that build the folded operand (then run the epilogue)
constexpr int kDefaultFoldWarps = 8;
constexpr int kMaxItems = 8;       // item ring depth (slab tile + folded operand)
constexpr int kBPerBlock = 4;      // consecutive |b| per block (one partial sum per group)
constexpr int kFoldCols = 32;      // tensor-memory columns per folded operand: 2 chunks x (hi, lo) x 8
constexpr int kSmemLimit = 227 * 1024;

// One ring item: the slab tiles of one (orbit, stage), hi then lo of each of
// its two 16-deep chunks; 8 bytes, so a block's item tables stay small.
struct __align__(8) TcItem {
  uint32_t off16;  // byte offset of the item's tiles in data, in 16-byte units
  uint8_t c16[2];  // accumulator column / 16 of each tile
  uint8_t n16[2];  // MMA N / 16 of each tile (0 = no tile)
  __host__ __device__ uint32_t col(int c) const { return 16u * c16[c]; }
  __host__ __device__ uint32_t n(int c) const { return 16u * n16[c]; }
  __host__ __device__ uint32_t bytes() const { return 64u * (n(0) + n(1)); }  // hi + lo of both tiles
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
  int in_lo = 0;          // input index of packed element 0
  int in_elems = 0;       // packed elements per position (32 * stages)
  int slot_bytes = 0;     // shared-memory slot per item
  int ring_pref = 0;      // item-ring depth chosen by oam_model_autotune (0 = deepest that fits)
  int tiling = 0;         // position tiling: 0 auto, 1 padded grid, 2 scan grid
  std::vector<double> row_cols;  // per |b|: MMA columns x 16 summed over a = 0 .. R and the stages
  int fold_warps = kDefaultFoldWarps;  // fold-warp count chosen by oam_model_autotune (4, 8 or 16)
  TcItem *d_items = nullptr;
  uint8_t *d_data = nullptr;
  size_t data_bytes = 0;
  CUtensorMap tmap;       // FP32 packed input [qtot][in_elems], box 32 x (128 + 2R), 128-byte swizzle
  CUtensorMap tmap_scan;  // the same with the scan-grid strip rows (when they fit one box)
};

}  // namespace oam

namespace {

struct CorrParams {
  long long qtot;
  int wp, px, py, R, W, stages;
  int sp;  // row stride of the grid the position tiles follow: Wp (padded) or px (scan)
  const int *tap_orbit;
  const TcItem *items;  // [n_orb][stages]
  const uint8_t *data;
  int slot_bytes, n_items, strip_rows, strip_bytes, items_bytes;
  int acc_cols, tmem_cols, fold_col0;
  float *part;         // partial sums [groups][py*px][acc_cols], one slice per group of kBPerBlock |b|
  size_t part_stride;  // py*px
  int *status;
  long long budget;
};

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(ptx::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(ptx::smem_addr(bar))
      : "memory");
}

// Does row offset `off` put any of the tile's rows inside the grid?
__device__ __forceinline__ bool row_live(const CorrParams &p, int tile, int off) {
  const int o0 = tile * kTileM, o1 = min(o0 + kTileM, p.py * p.sp) - 1;
  const int y_first = o0 / p.sp, y_last = o1 / p.sp;
  return !(y_last + off < 0 || y_first + off >= p.py);
}

// Lateral offset |a| of the j-th item of a stage.  Items alternate between
// the small and the large offsets (0, R, 1, R - 1, ...): the band, and with it
// the MMA width N, grows with the offset, so each pair of items costs about
// the same MMA time while its fold work is the same for every pair.
__device__ __forceinline__ int a_of(int j, int R) { return (j & 1) ? R - (j >> 1) : (j >> 1); }

// Index of the n-th set bit of mask (n counted from 0).
__device__ __forceinline__ int nth_set(unsigned mask, int n) {
  for (int i = 0; i < kBPerBlock; ++i)
    if ((mask >> i) & 1u) {
      if (n == 0) return i;
      --n;
    }
  return 0;
}

// Packed FP32 pairs (two lanes of one 64-bit register) and their arithmetic.
__device__ __forceinline__ uint64_t add_f32x2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t sub_f32x2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t pack_f32x2(float x, float y) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void unpack_f32x2(uint64_t v, float &x, float &y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}

// Staged FP32 rows are 128 bytes with the TMA's 128-byte swizzle: 16-byte
// chunk c of row r sits at chunk c ^ (r & 7).  Read the 8 elements of
// quarter q as four FP32 pairs.
__device__ __forceinline__ void load_row(const float *strip, int row, int q, uint64_t (&v)[4]) {
  const ulonglong2 *r2 = reinterpret_cast<const ulonglong2 *>(strip + row * 32);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const ulonglong2 u = r2[(2 * q + i) ^ (row & 7)];
    v[2 * i] = u.x;
    v[2 * i + 1] = u.y;
  }
}

// Add the 8 elements of quarter q of a staged row.
__device__ __forceinline__ void add_row(const float *strip, int row, int q, uint64_t (&v)[4]) {
  const ulonglong2 *r2 = reinterpret_cast<const ulonglong2 *>(strip + row * 32);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const ulonglong2 u = r2[(2 * q + i) ^ (row & 7)];
    v[2 * i] = add_f32x2(v[2 * i], u.x);
    v[2 * i + 1] = add_f32x2(v[2 * i + 1], u.y);
  }
}

// Split four FP32 pairs into BF16 pairs hi = bf16(v) and lo = bf16(v - hi),
// both rounded to nearest even; element 2e in the low half of word e.
__device__ __forceinline__ void split_bf16(const uint64_t (&v)[4], uint32_t (&hv)[4], uint32_t (&lv)[4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float x, y;
    unpack_f32x2(v[e], x, y);
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(x, y);
    const uint32_t hb = *reinterpret_cast<const uint32_t *>(&h2);
    const uint64_t lo = sub_f32x2(v[e], pack_f32x2(__uint_as_float(hb << 16), __uint_as_float(hb & 0xffff0000u)));
    float lx, ly;
    unpack_f32x2(lo, lx, ly);
    const __nv_bfloat162 l2 = __floats2bfloat162_rn(lx, ly);
    hv[e] = hb;
    lv[e] = *reinterpret_cast<const uint32_t *>(&l2);
  }
}

// Fold one item: F = P[m + R + a] + P[m + R - a] (P[m + R] alone for a = 0)
// for this thread's row m and its E of the stage's 32 K elements (8-element
// quarters q0 .. q0 + E/8 - 1), split into BF16 hi/lo words in the order the
// tensor-memory store takes them: E = 8: hi[4], lo[4]; E >= 16: per 16-deep
// chunk, hi[8] then lo[8].
template <int E>
__device__ __forceinline__ void fold_item(const float *X1, int m, int R, int a, int q0, uint32_t (&w)[E]) {
  constexpr int NQ = E / 8;
  uint64_t f[NQ][4];
#pragma unroll
  for (int i = 0; i < NQ; ++i) load_row(X1, m + R + a, q0 + i, f[i]);
  if (a > 0) {
#pragma unroll
    for (int i = 0; i < NQ; ++i) add_row(X1, m + R - a, q0 + i, f[i]);
  }
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    uint32_t hv[4], lv[4];
    split_bf16(f[i], hv, lv);
    const int hb = E == 8 ? 0 : 16 * (i >> 1) + 4 * (i & 1);  // word of the quarter's first hi pair
    const int lb = E == 8 ? 4 : hb + 8;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      w[hb + e] = hv[e];
      w[lb + e] = lv[e];
    }
  }
}

// Store one folded item into its tensor-memory slot (slot column 0 = chunk 0
// hi, 8 = chunk 0 lo, 16 = chunk 1 hi, 24 = chunk 1 lo; a column holds two
// BF16 K elements).
template <int E>
__device__ __forceinline__ void store_item(uint32_t slot_addr, int q0, const uint32_t (&w)[E]) {
  if constexpr (E == 8) {
    const uint32_t col = (uint32_t)(16 * (q0 >> 1) + 4 * (q0 & 1));
    uint32_t h[4] = {w[0], w[1], w[2], w[3]}, l[4] = {w[4], w[5], w[6], w[7]};
    ptx::tmem_st4(slot_addr + col, h);
    ptx::tmem_st4(slot_addr + col + 8u, l);
  } else if constexpr (E == 16) {
    ptx::tmem_st16(slot_addr + (uint32_t)(8 * q0), w);  // q0 = 2 * chunk
  } else {
    ptx::tmem_st32(slot_addr, w);
  }
}

template <int FW>
__global__ void __launch_bounds__(64 + 32 * FW, 1)
    k_corr_fold(const __grid_constant__ CUtensorMap tmap, const CorrParams p) {
  constexpr int kFoldWarps = FW;
  constexpr int kThreads = 64 + 32 * FW;
  constexpr int G = FW / 4;   // K groups per tensor-memory lane quarter
  constexpr int E = 32 / G;   // stage K elements folded per thread and item
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 128-byte-swizzled TMA destinations need 1024-byte alignment
  uint8_t *smem = smem_raw + ((1024u - (ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  // item ring: slab tile in shared memory + folded operand in tensor memory;
  // items go in pairs (the two taps of one fold pass), one set of barriers per pair
  const int K = p.n_items, KP = K / 2;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  uint64_t *strip_full = bars, *strip_empty = bars + 3;  // one pair per strip buffer
  uint64_t *acc_ready = bars + 6, *acc_full = bars + 7;
  uint64_t *slab_full = bars + 8, *fold_full = bars + 8 + KP, *item_empty = bars + 8 + 2 * KP;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + 512);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 516);
  volatile int *never = reinterpret_cast<volatile int *>(smem + 520);  // stays 0: waits that ignore abort
  TcItem *sitems = reinterpret_cast<TcItem *>(smem + 1024);           // [kBPerBlock][stages][R+1]: the group's items
  // Three strip buffers in rotation: stage gs stages its row y+b in buffer
  // gs % 3 (which then holds P = X(y+b) + X(y-b)) and its row y-b in buffer
  // (gs + 1) % 3, free again once P is formed, so stage gs + 1 reuses it and
  // the buffer stage gs - 1 held P.
  uint8_t *strips = smem + 1024 + p.items_bytes;                       // [3][strip_bytes]
  uint8_t *slots = strips + 3 * p.strip_bytes;                         // [K][slot_bytes]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x;
  const int grp = (int)blockIdx.y;  // |b| = kBPerBlock * grp + i: rows y + b and y - b
  const int R = p.R, NA = R + 1;    // a = 0 .. R
  unsigned live = 0;                // group members i whose rows meet the grid
  for (int i = 0; i < kBPerBlock; ++i) {
    const int b = kBPerBlock * grp + i;
    if (b <= R && (row_live(p, tile, b) || row_live(p, tile, -b))) live |= 1u << i;
  }
  const bool skip = live == 0;
  const int y0 = tile * kTileM / p.sp, x0 = tile * kTileM % p.sp;  // the tile's first position
  const long long qt = (long long)y0 * p.wp + x0;                  // its padded index
  const int total = __popc(live) * p.stages;  // strip stages of the block: live members in order, stages within
  const int L = p.strip_rows;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) {
      ptx::mbar_init(&strip_full[i], 1);
      ptx::mbar_init(&strip_empty[i], kFoldWarps);
    }
    ptx::mbar_init(acc_ready, kFoldWarps);
    ptx::mbar_init(acc_full, 1);
    for (int i = 0; i < KP; ++i) {
      ptx::mbar_init(&slab_full[i], 1);
      ptx::mbar_init(&fold_full[i], kFoldWarps);
      ptx::mbar_init(&item_empty[i], 1);
    }
    *abort_flag = 0;
    *never = 0;
    ptx::mbar_fence_init();
  }
  if (!skip) {  // the group's item tables [member][stage][item j], loaded by every thread in one pass
    const int n = p.stages * NA;
    for (int j = threadIdx.x; j < kBPerBlock * n; j += kThreads) {
      const int i = j / n, r = j % n, b = kBPerBlock * grp + i;
      if (!((live >> i) & 1u)) continue;
      const int st = r / NA, a = a_of(r % NA, R);
      sitems[j] = p.items[p.tap_orbit[(b + R) * p.W + (a + R)] * p.stages + st];
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
    if (lane == 0 && !skip) {
      int it_slab = 0;
      int uses[3] = {0, 0, 0};  // loads issued per strip buffer (one full / empty phase each)
      int k = 0;
      uint32_t lap = 0;  // parity of the item ring's current lap
      bool ok = true;
      // Block stage gs (member gs / stages, K stage gs % stages) loads row y+b
      // into buffer gs % 3 and row y-b into buffer (gs + 1) % 3 (a load of no
      // bytes for b = 0), each once the fold warps have released the buffer's
      // previous use.  The rows for stage gs + 1 are requested right after
      // stage gs's first slab tile, about a stage ahead of their use, instead
      // of after stage gs's last tile (which the item ring throttles to just
      // before the fold warps need the rows).
      auto load_strips = [&](int gs) {
        const int st = gs % p.stages;
        const int b = kBPerBlock * grp + nth_set(live, gs / p.stages);
        const int q_p = (int)((long long)(R + 1) * p.wp + qt + (long long)b * p.wp - R);
        const int q_m = (int)((long long)(R + 1) * p.wp + qt - (long long)b * p.wp - R);
        for (int r = 0; r < 2; ++r) {
          const int s = (gs + r) % 3;
          if (!ptx::mbar_wait(&strip_empty[s], (uses[s] & 1) ^ 1, abort_flag, p.budget)) return false;
          const bool load = r == 0 || b > 0;
          ptx::mbar_arrive_expect_tx(&strip_full[s], load ? (uint32_t)(L * 128) : 0u);
          if (load) tma_load_2d(strips + (size_t)s * p.strip_bytes, &tmap, kStageK * st, r == 0 ? q_p : q_m, &strip_full[s]);
          ++uses[s];
        }
        return true;
      };
      if (!load_strips(0)) {
        fail(1);
        ok = false;
      }
      for (int gs = 0; gs < total && ok; ++gs) {
        const TcItem *row_items = sitems + (nth_set(live, gs / p.stages) * p.stages + gs % p.stages) * NA;
        for (int a = 0; a < NA; a += 2) {  // pair slot k holds items a (slot 2k) and a + 1 (slot 2k + 1) of the stage
          const TcItem ia = row_items[a], ib = a + 1 < NA ? row_items[a + 1] : TcItem{};
          if (!ptx::mbar_wait(&item_empty[k], lap ^ 1, abort_flag, p.budget)) {
            fail(2);
            ok = false;
            break;
          }
          ptx::mbar_arrive_expect_tx(&slab_full[k], ia.bytes() + ib.bytes());
          if (ia.bytes() > 0)
            ptx::bulk_g2s(slots + (size_t)(2 * k) * p.slot_bytes, p.data + (size_t)ia.off16 * 16, ia.bytes(),
                          &slab_full[k]);
          if (ib.bytes() > 0)
            ptx::bulk_g2s(slots + (size_t)(2 * k + 1) * p.slot_bytes, p.data + (size_t)ib.off16 * 16, ib.bytes(),
                          &slab_full[k]);
          ++it_slab;
          if (++k == KP) {
            k = 0;
            lap ^= 1;
          }
          if (a == 0 && gs + 1 < total && !load_strips(gs + 1)) {
            fail(1);
            ok = false;
            break;
          }
        }
      }
      if (!ok) {
        // let copies already issued land before the block exits
        for (int i = std::max(0, it_slab - KP); i < it_slab; ++i)
          ptx::mbar_wait(&slab_full[i % KP], (i / KP) & 1, never, p.budget);
        for (int s = 0; s < 3; ++s)  // each buffer's last load (earlier ones were consumed before it was issued)
          if (uses[s] > 0) ptx::mbar_wait(&strip_full[s], (uses[s] - 1) & 1, never, p.budget);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // The whole warp walks the item ring, so every MMA operand is computed
    // warp-uniformly; one elected lane issues the MMAs and commits.  (A loop
    // run by a single lane issues at about half the rate.)
    bool ok = __all_sync(0xffffffffu, ptx::mbar_wait(acc_ready, 0, abort_flag, p.budget));
    if (!ok && lane == 0) fail(4);
    ptx::tc_fence_after();
    const bool leader = ptx::elect_one();
    int k = 0;
    uint32_t lap = 0;
    // B descriptor template (start-address field in 16-byte units; fields never carry)
    const uint64_t slot_desc = ptx::smem_desc(ptx::smem_addr(slots), 0, 128);
    const uint32_t idesc_m128 = ptx::idesc_bf16_f32(kTileM, 0);
    for (int gs = 0; gs < total && ok && !skip; ++gs) {
      const TcItem *row_items = sitems + (nth_set(live, gs / p.stages) * p.stages + gs % p.stages) * NA;
      for (int a = 0; a < NA; a += 2) {
        bool w = ptx::mbar_wait(&slab_full[k], lap, abort_flag, p.budget);
        if (w) w = ptx::mbar_wait(&fold_full[k], lap, abort_flag, p.budget);
        if (!__all_sync(0xffffffffu, w)) {
          if (lane == 0) fail(8);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        for (int h = 0; h < 2 && a + h < NA; ++h) {
          const TcItem item = row_items[a + h];
          const uint32_t slot = (uint32_t)(2 * k + h);
          const uint32_t a_base = tmem + (uint32_t)p.fold_col0 + 32u * slot;
          const uint64_t dB = slot_desc + (uint64_t)((slot * (uint32_t)p.slot_bytes) >> 4);
          const uint32_t n0 = item.n(0), n1 = item.n(1);
          const uint64_t b0h = dB + ((uint64_t)n0 << 16), b0l = b0h + 2u * n0;  // lbo = 16 n bytes; lo 32 n bytes on
          const uint64_t dB1 = dB + 4u * n0;                                   // second tile 64 n0 bytes later
          const uint64_t b1h = dB1 + ((uint64_t)n1 << 16), b1l = b1h + 2u * n1;
          const uint32_t i0 = idesc_m128 | ((n0 >> 3) << 17), i1 = idesc_m128 | ((n1 >> 3) << 17);
          const uint32_t d0 = tmem + item.col(0), d1 = tmem + item.col(1);
          if (leader) {
            // the two chunks accumulate into different columns: interleave them
            if (n0) ptx::mma_bf16_ta(d0, a_base, b0h, i0, 1);
            if (n1) ptx::mma_bf16_ta(d1, a_base + 16u, b1h, i1, 1);
            if (n0) ptx::mma_bf16_ta(d0, a_base + 8u, b0h, i0, 1);
            if (n1) ptx::mma_bf16_ta(d1, a_base + 24u, b1h, i1, 1);
            if (n0) ptx::mma_bf16_ta(d0, a_base, b0l, i0, 1);
            if (n1) ptx::mma_bf16_ta(d1, a_base + 16u, b1l, i1, 1);
          }
        }
        if (leader) ptx::mma_commit(&item_empty[k]);  // the pair's slots are free once its MMAs complete
        __syncwarp();
        if (++k == KP) {
          k = 0;
          lap ^= 1;
        }
      }
    }
    if (leader) ptx::mma_commit(acc_full);
    __syncwarp();
  } else {
    // ------------------------------------------------------------ fold warps, then epilogue
    const int fw = warp - 2;        // 0 .. kFoldWarps-1
    const int quarter = warp & 3;   // tensor-memory lanes 32*quarter .. +31
    const int kq = fw >> 2;         // K group of the stage this warp folds (E elements)
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    const int nb = (p.acc_cols + 31) / 32;  // 32-column blocks of the accumulator
    const int blk_begin = kq * nb / G, blk_end = (kq + 1) * nb / G;
    for (int j = blk_begin; j < blk_end; ++j) ptx::tmem_st32_zero(tmem + lane_base + (uint32_t)(32 * j));
    ptx::tmem_wait_st();
    ptx::tc_fence_before();
    __syncwarp();
    if (lane == 0) ptx::mbar_arrive(acc_ready);

    bool ok = true;
    if (!skip) {
      const int m = 32 * quarter + lane;  // row (tensor-memory lane) this thread folds
      const int om = tile * kTileM + m;
      const int pm = (om / p.sp - y0) * p.wp + (om % p.sp - x0);  // its padded offset from the tile's first
      const int q0 = kq * (E / 8);        // first 8-element quarter of the stage
      int uses[3] = {0, 0, 0}, k = 0;  // strip buffer uses consumed, as the producer counts them
      uint32_t lap = 0;
      for (int gs = 0; gs < total && ok; ++gs) {
        const int b = kBPerBlock * grp + nth_set(live, gs / p.stages);
        const int s = gs % 3, s2 = (gs + 1) % 3;
        ok = ptx::mbar_wait(&strip_full[s], uses[s] & 1, abort_flag, p.budget);
        if (ok) ok = ptx::mbar_wait(&strip_full[s2], uses[s2] & 1, abort_flag, p.budget);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          if (lane == 0) fail(32);
          break;
        }
        float *X1 = reinterpret_cast<float *>(strips + (size_t)s * p.strip_bytes);
        if (b > 0) {
          // P = X(y+b) + X(y-b) in place: both strips share the swizzle, so the
          // sum runs over physical float4s.
          const float4 *X2 = reinterpret_cast<const float4 *>(strips + (size_t)s2 * p.strip_bytes);
          float4 *P4 = reinterpret_cast<float4 *>(X1);
          for (int i = threadIdx.x - 64; i < L * 8; i += 32 * kFoldWarps) {
            float4 u = P4[i];
            const float4 v = X2[i];
            u.x += v.x;
            u.y += v.y;
            u.z += v.z;
            u.w += v.w;
            P4[i] = u;
          }
          asm volatile("bar.sync 1, %0;" ::"r"(32 * kFoldWarps) : "memory");  // fold warps only
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&strip_empty[s2]);  // row y-b is folded into P (or was not loaded)
        ++uses[s2];
        // two items (a, a + 1) per pass, in pair slot k: one wait, fence and barrier step for both
        for (int a = 0; a < NA; a += 2) {
          const bool two = a + 1 < NA;
          uint32_t w0[E], w1[E];  // folded in registers while the pair slot may still be in use
          fold_item<E>(X1, pm, R, a_of(a, R), q0, w0);
          if (two) fold_item<E>(X1, pm, R, a_of(a + 1, R), q0, w1);
          ok = ptx::mbar_wait(&item_empty[k], lap ^ 1, abort_flag, p.budget);
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) {
            if (lane == 0) fail(64);
            break;
          }
          const uint32_t fa = tmem + lane_base + (uint32_t)p.fold_col0 + 64u * (uint32_t)k;
          store_item<E>(fa, q0, w0);
          if (two) store_item<E>(fa + 32u, q0, w1);
          ptx::tmem_wait_st();
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&fold_full[k]);
          if (++k == KP) {
            k = 0;
            lap ^= 1;
          }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&strip_empty[s]);
        ++uses[s];
      }
    }

    // epilogue: this warp's lane quarter and column half of the accumulator
    bool done = ptx::mbar_wait(acc_full, 0, abort_flag, 4 * p.budget);
    done = __all_sync(0xffffffffu, done && ok);
    ptx::tc_fence_after();
    const int mrow = 32 * quarter + lane;
    const int o = tile * kTileM + mrow;  // this lane's position in the tile grid
    const int y = o / p.sp, x = o % p.sp;
    const bool valid = done && y < p.py && x < p.px;
    float *row = p.part + ((size_t)grp * p.part_stride + (size_t)y * p.px + x) * p.acc_cols;
    if (done) {
      for (int j = blk_begin; j < blk_end; ++j) {
        const int col = 32 * j;
        uint32_t r[32];
        ptx::tmem_ld32(tmem + lane_base + (uint32_t)col, r);
        ptx::tmem_wait_ld();
        if (valid) {
          float4 *dst = reinterpret_cast<float4 *>(row + col);
          const int nv = std::min(8, (p.acc_cols - col) >> 2);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < nv)
              dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                   __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
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

// Iterate in[py][px][len] -> out[qtot][elems] (FP32): element e of padded
// position q is index first + e of the row of (y, x) = (q / wp - R - 1, q % wp),
// zero outside the grid or the row.
__global__ void k_pack_input(const float *__restrict__ in, int len, int first, int elems, long long qtot, int wp,
                             int R, int px, int py, float4 *__restrict__ out) {
  const int e4n = elems >> 2;
  const long long total = qtot * e4n;
  const bool vec = ((len | first) & 3) == 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / e4n;
    const int e = 4 * (int)(i % e4n);
    const int y = (int)(q / wp) - (R + 1), x = (int)(q % wp);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (y >= 0 && y < py && x < px) {
      const float *src = in + ((size_t)y * px + x) * len;
      const int idx = first + e;
      if (vec && idx + 3 < len) {
        v = *reinterpret_cast<const float4 *>(src + idx);
      } else {
        if (idx < len) v.x = src[idx];
        if (idx + 1 < len) v.y = src[idx + 1];
        if (idx + 2 < len) v.z = src[idx + 2];
        if (idx + 3 < len) v.w = src[idx + 3];
      }
    }
    out[i] = v;
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

// Strip rows a block stages per row offset: 128 positions wrap at most
// (px + 126) / px scan rows, each adding R rows of padding to the span, plus
// R rows of halo on either side.
int strip_rows_for(int px, int R) { return kTileM + ((px + kTileM - 2) / px + 2) * R; }

// Executed MMA flops of one application: 3 products x 2 x M x (16 x N) over
// the (position tile, |b|, a >= 0) work items whose rows meet the grid, for
// position tiles along rows of stride sp.
double exec_flops_for(const oam_model *m, const TcLayout *L, int sp) {
  const int R = m->R, py = m->grid.py;
  const long long n_tiles = ((long long)py * sp + kTileM - 1) / kTileM;
  double total = 0;
  for (long long t = 0; t < n_tiles; ++t) {
    const long long yf = t * kTileM / sp, yl = (std::min(t * kTileM + kTileM, (long long)py * sp) - 1) / sp;
    for (int b = 0; b <= R; ++b) {
      const bool lp = !(yl + b < 0 || yf + b >= py), lm = !(yl - b < 0 || yf - b >= py);
      if (lp || lm) total += L->row_cols[b];
    }
  }
  return 3.0 * 2.0 * kTileM * total;
}

// Groups of kBPerBlock consecutive |b| = 0 .. R (the kernel's grid y, the partial sums).
int b_groups(int R) { return (R + 1 + kBPerBlock - 1) / kBPerBlock; }

int pow2_cols(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

oam_status encode_tmap(CUtensorMap *map, float *base, long long qtot, int elems, int rows) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return OAM_ERR_CUDA;
    }
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)elems, (cuuint64_t)qtot};
  const cuuint64_t strides[1] = {(cuuint64_t)elems * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kStageK, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  if (fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return OAM_ERR_CUDA;
  return OAM_OK;
}

// One direction's item and tile tables from the band form (host only).
oam_status plan_dir(const oam_model *m, TcLayout *L, int dir, std::vector<TcItem> &items,
                    std::vector<TcTile> &tiles) {
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
  L->in_elems = kStageK * L->stages;
  L->tmem_cols = pow2_cols(L->acc_cols);
  if (L->tmem_cols > 512) return OAM_ERR_UNSUPPORTED;

  items.assign((size_t)O * L->stages, TcItem{});
  tiles.clear();
  long long off = 0;
  int max_item = 16;
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
          it.c16[c] = 0;
          it.n16[c] = 0;
          continue;
        }
        const int col = lo & ~15;
        const int n = ((hi - col) + 15) & ~15;
        if (n > 256 || col + n > L->acc_cols) return OAM_ERR_UNSUPPORTED;
        it.c16[c] = (uint8_t)(col / 16);
        it.n16[c] = (uint8_t)(n / 16);
        tiles.push_back(TcTile{o, chunk, col, n, off});
        off += 64LL * n;  // hi + lo: 2 x (n rows x 16 elements x 2 bytes)
      }
      if (it.bytes() != (uint32_t)(off - item_off)) return OAM_ERR_DEVICE;  // the tiles are packed back to back
      max_item = std::max(max_item, (int)it.bytes());
      items[(size_t)o * L->stages + s] = it;
    }
  }
  L->slot_bytes = (max_item + 127) & ~127;
  L->data_bytes = (size_t)std::max<long long>(off, 16);
  // MMA columns per |b| (summed over a = 0 .. R); executed flops follow from
  // the tiles whose rows meet the grid (exec_flops_for)
  {
    std::vector<double> orb_cols(O, 0.0);
    for (const TcTile &t : tiles) orb_cols[t.orbit] += 16.0 * t.n;
    const int W = m->W, R = m->R;
    L->row_cols.assign(R + 1, 0.0);
    for (int b = 0; b <= R; ++b)
      for (int a = 0; a <= R; ++a) L->row_cols[b] += orb_cols[m->h_tap_orbit[(b + R) * W + (a + R)]];
  }
  return OAM_OK;
}

// Build one direction's item and tile tables from the band form, then pack.
oam_status build_dir(oam_model *m, TcLayout *L, int dir, cudaStream_t st, int *d_band_hi) {
  std::vector<TcItem> items;
  std::vector<TcTile> tiles;
  oam_status rc = plan_dir(m, L, dir, items, tiles);
  if (rc) return rc;
  const int nz = m->grid.nz, t_lo = m->n_lo & ~15;
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

struct Launch {
  CorrParams p;
  size_t smem;
  int tiling;   // 1 padded grid, 2 scan grid
  int n_tiles;  // position tiles (the grid's x)
};

oam_status plan_launch(const oam_model *m, const TcLayout *L, Launch *out) {
  const int R = m->R, px = m->grid.px, py = m->grid.py;
  CorrParams p{};
  p.qtot = m->tc_qtot;
  p.wp = px + R;
  p.px = px;
  p.py = py;
  p.R = R;
  p.W = m->W;
  p.stages = L->stages;
  p.tap_orbit = m->d_tap_orbit;
  p.items = L->d_items;
  p.data = L->d_data;
  p.slot_bytes = L->slot_bytes;
  p.items_bytes = (int)((sizeof(TcItem) * kBPerBlock * L->stages * (R + 1) + 1023) & ~size_t(1023));
  p.fold_col0 = (L->acc_cols + 31) & ~31;
  const int tmem_items = (512 - p.fold_col0) / kFoldCols;
  auto strip_bytes = [](int rows) { return (rows * 128 + 1023) & ~1023; };  // 128-byte rows, 1024-byte aligned
  auto fixed_for = [&](int rows) { return 1024 /* alignment slack */ + 1024 + p.items_bytes + 3 * strip_bytes(rows); };
  auto ring_for = [&](int rows) {  // deepest ring (whole pairs) that shared and tensor memory hold
    const int n = std::min(kMaxItems, std::min(tmem_items, (kSmemLimit - fixed_for(rows)) / L->slot_bytes));
    return n < 0 ? 0 : n & ~1;
  };
  const int rows_pad = kTileM + 2 * R, rows_scan = strip_rows_for(px, R);
  int tiling = L->tiling;
  if (tiling == 0)  // the scan grid unless its longer strips cost ring depth
    tiling = rows_scan <= 256 && ring_for(rows_scan) >= ring_for(rows_pad) ? 2 : 1;
  if (tiling == 2 && rows_scan > 256) return OAM_ERR_UNSUPPORTED;
  p.sp = tiling == 2 ? px : p.wp;
  p.strip_rows = tiling == 2 ? rows_scan : rows_pad;
  p.strip_bytes = strip_bytes(p.strip_rows);
  const int fixed = fixed_for(p.strip_rows);
  p.n_items = ring_for(p.strip_rows);
  if (L->ring_pref >= 2) p.n_items = std::min(p.n_items, L->ring_pref);
  p.n_items &= ~1;  // items go in pairs (one fold pass each)
  if (p.n_items < 2) return OAM_ERR_UNSUPPORTED;
  p.acc_cols = L->acc_cols;
  p.tmem_cols = 32;
  while (p.tmem_cols < p.fold_col0 + kFoldCols * p.n_items) p.tmem_cols <<= 1;
  p.part = m->d_tc_part;
  p.part_stride = (size_t)py * px;
  p.status = m->d_status;
  p.budget = 4000000000LL;  // ~2 s at 2 GHz
  out->p = p;
  out->smem = (size_t)fixed + (size_t)p.n_items * p.slot_bytes;
  out->tiling = tiling;
  out->n_tiles = (int)(((long long)py * p.sp + kTileM - 1) / kTileM);
  if (out->smem > (size_t)kSmemLimit) return OAM_ERR_UNSUPPORTED;
  return OAM_OK;
}

template <int FW>
oam_status launch_fold(const Launch &lp, const TcLayout *L, dim3 grid, cudaStream_t st) {
  OAM_CUDA_TRY(cudaFuncSetAttribute(k_corr_fold<FW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lp.smem));
  k_corr_fold<FW><<<grid, 64 + 32 * FW, lp.smem, st>>>(lp.tiling == 2 ? L->tmap_scan : L->tmap, lp.p);
  OAM_LAUNCHED();
  return OAM_OK;
}

oam_status run_corr(const oam_model *m, const TcLayout *L, const float *in, int in_len, float *out, int out_len,
                    cudaStream_t st) {
  if (!m->d_tc_part || !m->d_tc_pack) return OAM_ERR_UNSUPPORTED;
  Launch lp;
  oam_status rc = plan_launch(m, L, &lp);
  if (rc) return rc;
  const int R = m->R;
  {
    const long long total = m->tc_qtot * (L->in_elems / 4);
    const int blocks = (int)std::min<long long>((total + 255) / 256, 16LL * m->sm_count);
    k_pack_input<<<blocks, 256, 0, st>>>(in, in_len, L->in_lo, L->in_elems, m->tc_qtot, m->grid.px + R, R, m->grid.px,
                                         m->grid.py, reinterpret_cast<float4 *>(m->d_tc_pack));
    OAM_LAUNCHED();
  }
  {
    ProfScope prof(m, st, L->dir == 0);
    const dim3 grid(lp.n_tiles, b_groups(R));
    if (L->fold_warps == 4) rc = launch_fold<4>(lp, L, grid, st);
    else if (L->fold_warps == 16) rc = launch_fold<16>(lp, L, grid, st);
    else rc = launch_fold<8>(lp, L, grid, st);
    if (rc) return rc;
  }
  const size_t npos = (size_t)m->grid.py * m->grid.px;
  const int blocks = (int)std::min<size_t>((npos * out_len + 255) / 256, 16ull * m->sm_count);
  k_sum_parts<<<blocks, 256, 0, st>>>(m->d_tc_part, b_groups(R), npos, L->acc_cols, L->out_lo, out_len, out);
  OAM_LAUNCHED();
  return OAM_OK;
}

}  // namespace

// Device bytes tc_build allocates, from the planned bands (host only; no
// device call).  Fails like tc_build on shapes the kernels do not take.
oam_status oam::tc_plan_bytes(const oam_model *m, size_t *bytes) {
  if (kTileM + 2 * m->R > 256) return OAM_ERR_UNSUPPORTED;  // padded-grid strip rows per TMA box
  TcLayout Lf, La;
  std::vector<TcItem> items;
  std::vector<TcTile> tiles;
  size_t b = 0;
  for (int dir = 0; dir < 2; ++dir) {
    TcLayout *L = dir == 0 ? &Lf : &La;
    oam_status rc = plan_dir(m, L, dir, items, tiles);
    if (rc) return rc;
    Launch lp;
    if ((rc = plan_launch(m, L, &lp))) return rc;
    b += alloc_bytes<TcItem>(items.size()) + alloc_bytes<uint8_t>(L->data_bytes);
  }
  const int wp = m->grid.px + m->R;
  const long long qtot = (long long)(m->grid.py + 2 * m->R + 2) * wp + 256;
  if (qtot > 0x7fffffffLL) return OAM_ERR_UNSUPPORTED;
  b += alloc_bytes<uint8_t>((size_t)std::max(Lf.in_elems, La.in_elems) * qtot * sizeof(float));
  b += alloc_bytes<float>((size_t)b_groups(m->R) * m->grid.py * m->grid.px * std::max(Lf.acc_cols, La.acc_cols));
  *bytes = b;
  return OAM_OK;
}

oam_status oam::tc_build(oam_model *m, cudaStream_t st) {
  if (kTileM + 2 * m->R > 256) return OAM_ERR_UNSUPPORTED;  // padded-grid strip rows per TMA box
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
  if (m->tc_qtot > 0x7fffffffLL) return OAM_ERR_UNSUPPORTED;
  const int elems = std::max(m->tc_fwd->in_elems, m->tc_adj->in_elems);
  m->tc_pack_bytes = (size_t)elems * m->tc_qtot * sizeof(float);
  rc = dev_alloc(m, &m->d_tc_pack, m->tc_pack_bytes);
  if (rc) return rc;
  for (TcLayout *L : {m->tc_fwd, m->tc_adj}) {
    rc = encode_tmap(&L->tmap, reinterpret_cast<float *>(m->d_tc_pack), m->tc_qtot, L->in_elems, kTileM + 2 * m->R);
    if (rc) return rc;
    if (strip_rows_for(m->grid.px, m->R) <= 256) {
      rc = encode_tmap(&L->tmap_scan, reinterpret_cast<float *>(m->d_tc_pack), m->tc_qtot, L->in_elems,
                       strip_rows_for(m->grid.px, m->R));
      if (rc) return rc;
    }
    Launch lp;
    rc = plan_launch(m, L, &lp);
    if (rc) return rc;
  }
  // One partial per (position, |b| group): bounds the MMA results summed into
  // one tensor-memory accumulator; the parts are added in FP32 in a fixed order.
  const int acc = std::max(m->tc_fwd->acc_cols, m->tc_adj->acc_cols);
  rc = dev_alloc(m, &m->d_tc_part, (size_t)b_groups(m->R) * m->grid.py * m->grid.px * acc);
  if (rc) return rc;
  return OAM_OK;
}

void oam::tc_free(oam_model *m, cudaStream_t st) {
  for (TcLayout *L : {m->tc_fwd, m->tc_adj}) {
    if (!L) continue;
    if (L->d_items) cudaFreeAsync(L->d_items, st);
    if (L->d_data) cudaFreeAsync(L->d_data, st);
    delete L;
  }
  m->tc_fwd = m->tc_adj = nullptr;
  if (m->d_tc_pack) cudaFreeAsync(m->d_tc_pack, st);
  m->d_tc_pack = nullptr;
  if (m->d_tc_part) cudaFreeAsync(m->d_tc_part, st);
  m->d_tc_part = nullptr;
}

double oam::tc_exec_flops(const oam_model *m, int dir) {
  const TcLayout *L = dir == 0 ? m->tc_fwd : m->tc_adj;
  Launch lp;
  if (!L || plan_launch(m, L, &lp)) return 0.0;
  return exec_flops_for(m, L, lp.p.sp);
}

oam_status oam::forward_tc(const oam_model *m, const float *H, float *s, cudaStream_t st) {
  return run_corr(m, m->tc_fwd, H, m->grid.nz, s, m->grid.nt, st);
}

oam_status oam::adjoint_tc(const oam_model *m, const float *s, float *H, cudaStream_t st) {
  return run_corr(m, m->tc_adj, s, m->grid.nt, H, m->grid.nz, st);
}

// ---------------------------------------------------------------- autotuner
// Per direction, time every (position tiling, fold-warp count, ring depth) on
// the model's own shapes (CUDA events on `st`) and keep the fastest.
oam_status oam::tc_autotune(oam_model *m, int reps, cudaStream_t st, int *best_fwd, int *best_adj, int *warps_fwd,
                            int *warps_adj) {
  if (!m->tc_fwd) return OAM_ERR_UNSUPPORTED;
  const size_t nv = vol_elems(m), ns = sig_elems(m);
  float *buf = nullptr;
  if (cudaMalloc((void **)&buf, (nv + ns) * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return OAM_ERR_OOM;
  }
  oam_status rc = OAM_OK;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemsetAsync(buf, 0, (nv + ns) * sizeof(float), st);
  for (int dir = 0; dir < 2 && !rc; ++dir) {
    TcLayout *L = dir == 0 ? m->tc_fwd : m->tc_adj;
    float best_ms = 1e30f;
    int best = 0, best_w = kDefaultFoldWarps, best_t = 0;
    for (int tiling = 1; tiling <= 2 && !rc; ++tiling) {
      L->tiling = tiling;
      L->ring_pref = 0;
      Launch lp;
      if (plan_launch(m, L, &lp)) continue;  // this tiling does not fit the model
      const int deepest = lp.p.n_items;
      for (int fw : kFoldWarpChoices) {
        L->fold_warps = fw;
        for (int depth = 2; depth <= deepest; depth += 2) {
          L->ring_pref = depth;
          for (int r = 0; r <= reps && !rc; ++r) {  // first run warms up
            if (r == 1) cudaEventRecord(e0, st);
            rc = dir == 0 ? run_corr(m, L, buf, m->grid.nz, buf + nv, m->grid.nt, st)
                          : run_corr(m, L, buf + nv, m->grid.nt, buf, m->grid.nz, st);
          }
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) rc = OAM_ERR_CUDA;
          if (rc) break;
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best_ms) {
            best_ms = ms;
            best = depth;
            best_w = fw;
            best_t = tiling;
          }
        }
        if (rc) break;
      }
    }
    L->tiling = best_t;
    L->ring_pref = best;
    L->fold_warps = best_w;
    (dir == 0 ? *best_fwd : *best_adj) = best;
    (dir == 0 ? *warps_fwd : *warps_adj) = best_w;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  return rc;
}

oam_status oam::tc_set_tiles(oam_model *m, int dir, int fold_warps, int ring) {
  TcLayout *L = dir == 0 ? m->tc_fwd : m->tc_adj;
  if (!L) return OAM_ERR_UNSUPPORTED;
  bool okw = false;
  for (int fw : kFoldWarpChoices) okw = okw || fw == fold_warps;
  if (!okw || ring < 0 || (ring & 1)) return OAM_ERR_INVALID_ARG;
  const int keep_ring = L->ring_pref, keep_w = L->fold_warps;
  L->ring_pref = ring;
  L->fold_warps = fold_warps;
  Launch lp;
  oam_status rc = plan_launch(m, L, &lp);
  if (rc || (ring >= 2 && lp.p.n_items != ring)) {
    L->ring_pref = keep_ring;
    L->fold_warps = keep_w;
    return rc ? rc : OAM_ERR_INVALID_ARG;
  }
  return OAM_OK;
}

oam_status oam::tc_set_tiling(oam_model *m, int dir, int tiling) {
  TcLayout *L = dir == 0 ? m->tc_fwd : m->tc_adj;
  if (!L) return OAM_ERR_UNSUPPORTED;
  if (tiling < 0 || tiling > 2) return OAM_ERR_INVALID_ARG;
  const int keep = L->tiling;
  L->tiling = tiling;
  Launch lp;
  const oam_status rc = plan_launch(m, L, &lp);
  if (rc) L->tiling = keep;
  return rc;
}

int oam::tc_get_tiling(const oam_model *m, int dir) {
  const TcLayout *L = dir == 0 ? m->tc_fwd : m->tc_adj;
  Launch lp;
  return L && plan_launch(m, L, &lp) == OAM_OK ? lp.tiling : 0;
}

void oam::tc_get_tiles(const oam_model *m, int dir, int *fold_warps, int *ring) {
  const TcLayout *L = dir == 0 ? m->tc_fwd : m->tc_adj;
  if (!L) {
    *fold_warps = *ring = 0;
    return;
  }
  Launch lp;
  *fold_warps = L->fold_warps;
  *ring = plan_launch(m, L, &lp) == OAM_OK ? lp.p.n_items : 0;
}
