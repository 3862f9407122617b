// The O(L^3) contractions on the tcgen05 tensor cores (3xTF32 split products, FP32 accumulation
// in tensor memory), for batched transforms.
//
// For each m >= 0 both signs of m share one matrix (eqn wignerd_sym6 gives
// Delta^l_{m',-m} = (-1)^{l+m'} Delta^l_{m'm}):
//   A_m[m', l] = U_l[m'] Delta^l_{m'm},   U_l[m'] = sqrt((2l+1)/4pi) Delta^l_{m',-s},
// nonzero for l >= max(m, m', |s|).  With columns j = (sign, part, b) over 4B real columns:
//   inverse (eqn fourier_coeff):  D[m', j] = sum_l A_m[m', l] V_m[l, j],
//       V_m[l, (0, part, b)] = part(sf_{l,m}[b]),  V_m[l, (1, part, b)] = (-1)^l part(sf_{l,-m}[b]);
//       F_{m m'} = (-1)^s i^{-(m+s)} D[m', (0, ., b)],  F_{-m, m'} = (-1)^s i^{m-s} (-1)^{m'} D[m', (1, ., b)].
//   forward / adjoint projection:  P[l, j] = sum_{m'} A_m[m', l] Y_m[m', j],
//       Y_m[m', (0, part, b)] = part(H_{m m'}[b]),  Y_m[m', (1, part, b)] = (-1)^{m'} part(H_{-m m'}[b]);
//       sf_{lm} = (-1)^s i^{m+s} P[l, (0, ., b)],  sf_{l,-m} = (-1)^s i^{-m+s} (-1)^l P[l, (1, ., b)].
// So every m is a real GEMM with M = 128-row blocks of m' (inverse) or l (forward), K = l or m'
// in chunks of 32, N = 2H columns, H = 2B rounded up to 16 (column sign*H + 2b + part).  Operands
// are split x = hi + lo (TF32) and the product is hi*hi + hi*lo + lo*hi (the dropped lo*lo is
// ~2^-22 relative).
//
// Accumulation.  The tensor core's FP32 accumulation truncates (rounds toward zero); over the
// 384 accumulation steps of K = 1024 that bias alone reaches ~1e-5 relative.  So each K chunk
// accumulates into a fresh tensor-memory segment, the two small correction products first and the
// four hi*hi products last (truncation then acts on four large steps only), and the epilogue warps
// add every segment into FP32 running sums in registers (round to nearest).
//
// Operands are written once per call (A also once per plan with the Delta cache) as tiles already
// in the K-major SWIZZLE_128B layout -- 3xTF32: the FP32 values (16 KB an A tile), split into hi and
// lo in shared memory when they arrive; split-BF16: both parts -- so the main kernel moves them with
// 1-D bulk copies.  Main kernel: persistent, one CTA per SM, 10 warps: warp 0 lane 0 issues the bulk
// copies (a ring of 2-4 stages), warp 1 lane 0 issues tcgen05.mma into one of two 128 x 256 FP32 accumulator
// segments in tensor memory, warps 2-9 (two per 32-lane quarter of tensor memory, one for each
// sign of m) read the accumulator with tcgen05.ld, apply the phases and write the outputs (the
// inverse writes half rows m' >= 0 of F; the torus passes apply the extension).  Work items (m, row
// block) are sorted (groups of four m, or decreasing length) and dealt to the CTAs by a greedy
// schedule made on the host (schedule()).  Every wait is bounded; a
// timeout latches a status bit and the CTA drains its copies and MMAs before leaving.
#include "ssht_internal.h"
#include "bounds.cuh"
#include "f32_round.h"
#include "tc_common.cuh"

#include <algorithm>
#include <queue>
#include <vector>

namespace ssht {
namespace {

using namespace tc;

constexpr int TM = kTileRows;              // rows per tile
constexpr int TK = kTileK;                 // K per chunk (one 128-byte TF32 row)
constexpr int A_PART = kAPart;             // 16 KB: one split part of an A tile
constexpr int A_TILE = kATile;             // both parts of an A tile in shared memory (hi then lo)
constexpr int MAX_STAGES = 4;             // pipeline depth: a plan parameter, 2 .. MAX_STAGES
constexpr int EPI_WARPS = 8;                       // two per tensor-memory lane quarter
constexpr int THREADS = 64 + 32 * EPI_WARPS;       // producer warp, MMA warp, epilogue warps

__host__ __device__ inline long long tri_ll(long long m) { return m * (m + 1) / 2; }
__host__ __device__ inline size_t doff(long long l) { return (size_t)(l * (l + 1) * (2 * l + 1) / 6); }

struct Item {
  int m, i, c0, c1;     // row block i of m; K chunks [c0, c1)
  long long atile;      // index of the A tile of chunk c0
};

struct TcArgs {
  int L, s, B, NC;        // B: fields of this slice; NC = 2H: padded columns, H = 2 Bs rounded up to 16 (<= 128)
  int stages;             // pipeline depth
  const int* sched;       // CTA b runs items [sched[b], sched[b + 1]) in order
  const Item* items;
  const uint8_t* A;       // packed A tiles
  const uint8_t* X;       // packed data tiles
  const long long* xoff;  // per m: data tile index of chunk xc0(m)
  const int* xc0;         // per m: first chunk stored for m
  const float2* ph;       // e^{i pi k/N}, k in [-(N-1), N-1], at k + N - 1
  float2* out;            // inverse: theta-DFT input E [B][N][N]; forward: flm [B][L*L]
  int* status;
  long long wait_ns;      // spin limit of the pipeline waits
  long long a_tiles, x_tiles, out_n;  // extents of A, this slice's data tiles and out (index checks)
};

__device__ __forceinline__ float2 ipow_signed(int s, int k) {
  const int r = ((k % 4) + 4) % 4;
  float a = (r == 0) ? 1.f : (r == 2) ? -1.f : 0.f;
  float b = (r == 1) ? 1.f : (r == 3) ? -1.f : 0.f;
  if (s & 1) { a = -a; b = -b; }
  return make_float2(a, b);
}

// ---------------------------------------------------------------------------------------------
// Packing: A tiles from the FP64 Delta table
// ---------------------------------------------------------------------------------------------

// Inverse A tile (m, i, c): rows m' = 128 i + r, columns l = 32 c + k (K-major).
// Forward A tile (m, i, c): rows l = 128 i + r, columns m' = 32 c + k.
// Every thread issues its 16 table loads before converting any of them.
template <bool FWD, bool BF>
__global__ void __launch_bounds__(256) pack_a_kernel(int L, int s, const Item* __restrict__ items,
                                                     const double* __restrict__ table, const float* __restrict__ Uf,
                                                     uint8_t* __restrict__ A, long long a_tiles) {
  __shared__ __align__(16) uint8_t tile[A_TILE];
  constexpr int PER = TM * TK / 256;
  const Item it = items[blockIdx.y];
  const int c = it.c0 + blockIdx.x;
  if (c >= it.c1) return;
  const int m = it.m, Lp = L - 1, as = s < 0 ? -s : s;
  double d[PER];
  float u[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = threadIdx.x + q * 256;
    const int r = FWD ? e / TK : e % TM, k = FWD ? e % TK : e / TM;
    const int rowv = it.i * TM + r, colv = c * TK + k;
    const int mp = FWD ? colv : rowv, l = FWD ? rowv : colv;
    const bool ok = l <= Lp && mp <= Lp && l >= m && l >= mp && l >= as;
    // Delta^l_{m' m} = (-1)^{m'-m} Delta^l_{m m'}: row m of degree l, contiguous in m'
    const long long ti = (long long)doff(l) + (long long)m * (l + 1) + mp, ui = (long long)tri_ll(l) + mp;
    d[q] = (ok && in_bounds(ti, (long long)doff(L), kbPackAIn)) ? __ldg(&table[ti]) : 0.0;
    u[q] = (ok && in_bounds(ui, (long long)tri_ll(L), kbPackAIn)) ? __ldg(&Uf[ui]) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = threadIdx.x + q * 256;
    const int r = FWD ? e / TK : e % TM, k = FWD ? e % TK : e / TM;
    const int mp = FWD ? c * TK + k : it.i * TM + r;
    const float a = u[q] * f64_to_f32_rn(d[q]);
    put_split<BF>(tile, A_PART, r, k, ((mp - m) & 1) ? -a : a);
  }
  __syncthreads();
  if (!in_bounds(it.atile + blockIdx.x, a_tiles, kbPackAOut)) return;
  constexpr int GA = kParts<BF> * A_PART;  // bytes of a tile in global memory
  uint4* dst = (uint4*)(A + (size_t)(it.atile + blockIdx.x) * GA);
  const uint4* src = (const uint4*)tile;
  for (int e = threadIdx.x; e < GA / 16; e += blockDim.x) dst[e] = src[e];
}

// ---------------------------------------------------------------------------------------------
// Packing: data tiles (rows j = (sign, part, b), K-major over 32 l or m')
// ---------------------------------------------------------------------------------------------

// Inverse data tiles (m, c): V_m[l, j], l = 32 c + k, rows j = sign * NC/2 + 2b (real part) and
// 2b + 1 (imaginary part), for 16 consecutive m at once.  For every field the coefficients
// sf_{l,+-m} of the 32 degrees of chunk c are read as runs of 16 consecutive orders (coalesced),
// turned around in shared memory, and every tile row -- 32 consecutive K = l -- is written by one
// warp at once; the rows of padding fields are written as zeros.  Fields run in slices of Bs
// (blockIdx.z): slice z holds fields z Bs .. z Bs + Bs - 1 in its own tile region of xslice bytes.
template <bool BF>
__global__ void __launch_bounds__(256) pack_v_kernel(int L, int s, int Btot, int Bs, size_t xslice, int NC,
                                                     const int* __restrict__ xc0, const long long* __restrict__ xoff,
                                                     const float2* __restrict__ flm, uint8_t* __restrict__ X) {
  __shared__ float2 sv[32][33];
  const int B = min(Bs, Btot - (int)blockIdx.z * Bs);
  const long long flm_n = (long long)Btot * L * L, flm0 = (long long)blockIdx.z * Bs * L * L;
  const long long x_tiles = (long long)(xslice / (kParts<BF> * (size_t)NC * 128));
  flm += (size_t)blockIdx.z * Bs * L * L;
  X += (size_t)blockIdx.z * xslice;
  const int c = blockIdx.x, m0 = 16 * blockIdx.y;
  // xc0 grows with m: when chunk c is below the first stored chunk of m0, no tile of this CTA's 16
  // orders is stored (about half the grid: the degrees of chunk c all lie below m0)
  if (m0 >= L || c < xc0[m0]) return;
  const int as = s < 0 ? -s : s;
  const int part_bytes = NC * 128, half = NC / 2, nb = half / 2;  // nb: fields of a sign half, padded
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int b = 0; b < nb; ++b) {
    if (b < B) {
      // 32 degrees l x (orders m0 .. m0 + 15, then -m0 .. -m0 - 15)
      for (int q = threadIdx.x; q < 1024; q += 256) {
        const int lo = q >> 5, col = q & 31, sign = col >> 4, m = m0 + (col & 15);
        const int l = c * TK + lo;
        float2 v = make_float2(0.f, 0.f);
        const long long fi = (long long)b * L * L + (long long)l * l + l + (sign ? -m : m);
        if (m < L && l < L && l >= m && l >= as && !(sign && m == 0) && in_bounds(flm0 + fi, flm_n, kbPackVIn)) {
          v = flm[fi];
          if (sign && (l & 1)) v = make_float2(-v.x, -v.y);
        }
        sv[lo][col] = v;
      }
    }
    __syncthreads();
    for (int cb = warp; cb < 32; cb += 8) {
      const int sign = cb >> 4, m = m0 + (cb & 15);
      if (m >= L || c < xc0[m]) continue;  // tile (m, c) is not stored
      if (!in_bounds(xoff[m] + (c - xc0[m]), x_tiles, kbPackVOut) || !in_bounds(sign * half + 2 * b + 1, NC, kbPackVOut))
        continue;
      uint8_t* tile = X + (size_t)(xoff[m] + (c - xc0[m])) * kParts<BF> * part_bytes;
      const float2 v = b < B ? sv[lane][cb] : make_float2(0.f, 0.f);
      const int j = sign * half + 2 * b;
      put_split<BF>(tile, part_bytes, j, lane, v.x);
      put_split<BF>(tile, part_bytes, j + 1, lane, v.y);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// The tensor-core GEMM
// ---------------------------------------------------------------------------------------------

// Loads 4 groups of 16 columns (64 values) of this warp's 32 tensor-memory lanes, one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
  uint32_t r[64];
#pragma unroll
  for (int g = 0; g < 4; ++g)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[16 * g + 0]), "=r"(r[16 * g + 1]), "=r"(r[16 * g + 2]), "=r"(r[16 * g + 3]),
                   "=r"(r[16 * g + 4]), "=r"(r[16 * g + 5]), "=r"(r[16 * g + 6]), "=r"(r[16 * g + 7]),
                   "=r"(r[16 * g + 8]), "=r"(r[16 * g + 9]), "=r"(r[16 * g + 10]), "=r"(r[16 * g + 11]),
                   "=r"(r[16 * g + 12]), "=r"(r[16 * g + 13]), "=r"(r[16 * g + 14]), "=r"(r[16 * g + 15])
                 : "r"(taddr + 16 * g));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 64; ++k) v[k] = __uint_as_float(r[k]);
}

template <bool FWD, bool BF>
__global__ void __launch_bounds__(THREADS, 1) tc_gemm_kernel(TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int b_part = a.NC * 128;
  const int stage_bytes = A_TILE + 2 * b_part;  // both split parts of A and of the data tile
  constexpr int GA = kParts<BF> * A_PART;       // bytes of an A tile in global memory
  const int gx = kParts<BF> * b_part;           // bytes of a data tile in global memory
  const int STAGES = a.stages;
  // full: a stage's copies have landed; ready (3xTF32): its FP32 values are split into hi + lo
  __shared__ __align__(8) uint64_t full[MAX_STAGES], ready[MAX_STAGES], empty[MAX_STAGES], seg_full[2], seg_empty[2],
      done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 1) tmem_alloc(&tmem_base, 512);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], EPI_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&seg_full[k], 1);
      mbar_init(&seg_empty[k], EPI_WARPS);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = tmem_base;
  volatile int* abort = &abort_flag;
  const int nC = (a.L + TK - 1) / TK;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: bulk copies of the A and data tiles of every chunk ----
      int it = 0;
      int last_use[MAX_STAGES] = {-1, -1, -1, -1};
      for (int w = a.sched[blockIdx.x]; w < a.sched[blockIdx.x + 1] && !*abort; ++w) {
        const Item itm = a.items[w];
        const uint8_t* Ab = a.A + (size_t)itm.atile * GA;
        for (int c = itm.c0; c < itm.c1; ++c, ++it) {
          const int s = it % STAGES, u = it / STAGES;
          if (!mbar_wait(&empty[s], (u & 1) ^ 1, abort, a.wait_ns)) {
            *abort = 1;
            break;
          }
          uint8_t* st = smem + s * stage_bytes;
          mbar_expect_tx(&full[s], (uint32_t)(GA + gx));
          // a tile index outside its array is recorded and tile 0 copied instead (the pipeline
          // still completes; the result is wrong and the record says why)
          const long long at = itm.atile + (c - itm.c0);
          const uint8_t* asrc = in_bounds(at, a.a_tiles, kbGemmA) ? Ab + (size_t)(c - itm.c0) * GA : a.A;
          bulk_g2s(st, asrc, GA, &full[s]);
          long long xt = FWD ? (long long)itm.m * nC + c : a.xoff[itm.m] + (c - a.xc0[itm.m]);
          if (!in_bounds(xt, a.x_tiles, kbGemmX)) xt = 0;
          bulk_g2s(st + A_TILE, a.X + (size_t)xt * gx, (uint32_t)gx, &full[s]);
          last_use[s] = u;
        }
      }
      // drain: every issued copy must have landed before the CTA leaves
      for (int s = 0; s < STAGES; ++s)
        if (last_use[s] >= 0) mbar_wait(&full[s], last_use[s] & 1, nullptr, kDrainNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: one tensor-memory segment per chunk, corrections first ----
      const uint32_t idesc = BF ? idesc_bf16(TM, a.NC) : idesc_tf32(TM, a.NC);
      int it = 0;
      for (int w = a.sched[blockIdx.x]; w < a.sched[blockIdx.x + 1] && !*abort; ++w) {
        const Item itm = a.items[w];
        bool ok = true;
        for (int c = itm.c0; c < itm.c1; ++c, ++it) {
          const int s = it % STAGES, u = it / STAGES;
          const int seg = it & 1, us = it >> 1;
          if (!mbar_wait(&seg_empty[seg], (us & 1) ^ 1, abort, a.wait_ns) ||
              !mbar_wait(BF ? &full[s] : &ready[s], u & 1, abort, a.wait_ns)) {
            *abort = 1;
            ok = false;
            break;
          }
          fence_after();
          const uint32_t dt = tbase + (uint32_t)(seg * 256);
          const uint32_t sa = smem_u32(smem + s * stage_bytes);
          const uint32_t sb = sa + A_TILE;
          if constexpr (BF) {
            // parts h, m at bytes 0 and 64 of part 0, l at byte 0 of part 1; K = 16 (32 bytes)
            // per instruction.  Products from the smallest up: h*l, l*h, m*m, h*m, m*h, h*h.
            const uint32_t oa[3] = {0u, 64u, (uint32_t)A_PART}, ob[3] = {0u, 64u, (uint32_t)b_part};
            const int pa[6] = {0, 2, 1, 0, 1, 0}, pb[6] = {2, 0, 1, 1, 0, 0};
#pragma unroll
            for (int q = 0; q < 6; ++q)
#pragma unroll
              for (int kk = 0; kk < 2; ++kk)
                mma_bf16(dt, desc_sw128(sa + oa[pa[q]] + kk * 32), desc_sw128(sb + ob[pb[q]] + kk * 32), idesc,
                         (q == 0 && kk == 0) ? 0u : 1u);
          } else {
#pragma unroll
            for (int kk = 0; kk < TK / 8; ++kk) {
              const uint32_t ko = kk * 32;
              mma_tf32(dt, desc_sw128(sa + ko), desc_sw128(sb + b_part + ko), idesc, kk == 0 ? 0u : 1u);  // hi * lo
              mma_tf32(dt, desc_sw128(sa + A_PART + ko), desc_sw128(sb + ko), idesc, 1u);                 // lo * hi
            }
#pragma unroll
            for (int kk = 0; kk < TK / 8; ++kk) {
              const uint32_t ko = kk * 32;
              mma_tf32(dt, desc_sw128(sa + ko), desc_sw128(sb + ko), idesc, 1u);                          // hi * hi
            }
          }
          mma_commit(&empty[s]);
          mma_commit(&seg_full[seg]);
        }
        if (!ok) break;
      }
      mma_commit(&done_bar);
      mbar_wait(&done_bar, 0, nullptr, kDrainNs);  // every issued MMA has completed
    }
  } else {
    // ---- epilogue: running sums of the segments, then phases and outputs ----
    const int q = warp & 3;                // tensor-memory lane quarter this warp may access
    const int h = (warp - 2) >> 2;         // column half: sign of m
    const int r = q * 32 + lane;
    const int L = a.L, Lp = L - 1, NT = 2 * L - 1, B = a.B, s = a.s;
    const int H = a.NC / 2;
    const uint32_t tq = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * H);
    // 3xTF32: the epilogue warps also split each arrived stage's FP32 values into hi + lo, one
    // chunk ahead of the chunk they sum, so that the split of chunk c + 1 overlaps the MMAs of c
    int nchunks = 0, conv = 0;
    if constexpr (!BF)
      for (int w = a.sched[blockIdx.x]; w < a.sched[blockIdx.x + 1]; ++w) nchunks += a.items[w].c1 - a.items[w].c0;
    const int et = threadIdx.x - 64, ent = 32 * EPI_WARPS;
    auto convert_upto = [&](int last) -> bool {
      for (; conv < nchunks && conv <= last; ++conv) {
        const int sc = conv % STAGES, uc = conv / STAGES;
        if (!mbar_wait(&full[sc], uc & 1, abort, a.wait_ns)) return false;
        uint8_t* st = smem + sc * stage_bytes;
        split_region_tf32(st, A_PART, A_PART, et, ent);
        split_region_tf32(st + A_TILE, b_part, b_part, et, ent);
        fence_proxy_async();  // the split parts are read by the tensor core (async proxy)
        __syncwarp();
        if (lane == 0) mbar_arrive(&ready[sc]);
      }
      return true;
    };
    int it = 0;
    for (int w = a.sched[blockIdx.x]; w < a.sched[blockIdx.x + 1] && !*abort; ++w) {
      const Item itm = a.items[w];
      float acc[128];
#pragma unroll
      for (int k = 0; k < 128; ++k) acc[k] = 0.f;
      bool ok = true;
      for (int c = itm.c0; c < itm.c1; ++c, ++it) {
        const int seg = it & 1, us = it >> 1;
        if constexpr (!BF) {
          if (!convert_upto(it + 1)) {
            *abort = 1;
            ok = false;
            break;
          }
        }
        if (!mbar_wait(&seg_full[seg], us & 1, abort, a.wait_ns)) {
          *abort = 1;
          ok = false;
          break;
        }
        fence_after();
        const uint32_t ts = tq + (uint32_t)(seg * 256);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          if (64 * g < H) {
            float v[64];
            tmem_ld64(ts + 64 * g, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) acc[64 * g + k] += v[k];
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&seg_empty[seg]);
      }
      if (!ok) break;
      const int m = itm.m;
      if (h == 1 && m == 0) continue;
      const int rowv = itm.i * TM + r;  // m' (inverse) or l (forward)
      const bool valid = FWD ? (rowv <= Lp && rowv >= m) : (rowv <= Lp);
      if (!valid) continue;
      const int mm = h ? -m : m;
      const float2 pz = FWD ? ipow_signed(s, mm + s) : ipow_signed(s, -(mm + s));
      const float rs = (h && (rowv & 1)) ? -1.f : 1.f;  // (-1)^{m'} (inverse) or (-1)^l (forward) for -m
#pragma unroll
      for (int b = 0; b < 64; ++b) {
        if (b >= B) break;
        const float xr = rs * acc[2 * b], xi = rs * acc[2 * b + 1];
        const float2 F = make_float2(pz.x * xr - pz.y * xi, pz.x * xi + pz.y * xr);
        const long long o = FWD ? (long long)b * L * L + (long long)rowv * rowv + rowv + mm
                                : ((long long)b * NT + (mm + Lp)) * L + rowv;  // half row m' >= 0
        if (in_bounds(o, a.out_n, kbGemmOut)) a.out[o] = F;
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (*abort && threadIdx.x == 0) atomicOr(a.status, 2);
  if (warp == 1) tmem_dealloc(tbase, 512);
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------

struct TcPlan {
  int L = 0, s = 0, B = 0, NC = 0, nC = 0, nI = 0;
  bool bf16 = false;  // split-BF16 (3 parts, 6 products) instead of 3xTF32
  TcConfig cfg;
  int Bs = 0, nS = 0;        // fields per slice (one GEMM launch each) and slices
  size_t xslice = 0;         // bytes of one slice's data tiles
  std::vector<Item> inv_h, fwd_h;  // work items in creation order (re-sorted by the configuration)
  Item* items_inv = nullptr;  // in schedule order: CTA-major
  Item* items_fwd = nullptr;
  int* sched_inv = nullptr;   // per CTA: first item (grid + 1 entries)
  int* sched_fwd = nullptr;
  int grid_inv = 0, grid_fwd = 0;
  int n_inv = 0, n_fwd = 0;
  long long tiles_A = 0, tiles_inv = 0, xtiles_inv = 0, xtiles_fwd = 0;
  // Forward A tiles (m, i, c): rows l = 128 i + r, K = m' = 32 c + k, tile index abase[m] +
  // 2i(i+1) - 2 i_m(i_m+1) + c with i_m = m / 128 (each (m, i), i >= i_m, holds 4i + 4 slots;
  // entries nothing writes stay zero).  Inverse A tiles A_inv (m, i, c): rows m' = 128 i + r,
  // K = l = 32 c + k, at the item's tile index.  Both are shared by every slice of fields.
  uint8_t* A = nullptr;
  uint8_t* A_inv = nullptr;
  long long* abase = nullptr;
  long long* ibase = nullptr;  // [m * nI + i]: tile index of chunk kc of inverse item (m, i) is ibase + kc
  uint8_t* X = nullptr;        // data tiles, nS slices of xslice bytes
  size_t xbytes = 0;
  long long* xoff = nullptr;
  int* xc0 = nullptr;
  size_t bytes = 0;
  int grid = 0;
  size_t smem = 0;
  int smem_max = 0;
};

static cudaError_t tc_alloc(void** p, size_t bytes, size_t* total) {
  cudaError_t e = dev_malloc(p, bytes ? bytes : 16);
  if (e == cudaSuccess) *total += bytes;
  return e;
}

template <class K>
static cudaError_t gemm_attrs(K kernel, int bytes) {
  cudaError_t e = prefer_shared(kernel);
  return e != cudaSuccess ? e : cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

static int nc_of(int Bs) { return 2 * (((2 * Bs + 15) / 16) * 16); }
static size_t stage_bytes_of(int NC) { return (size_t)A_TILE + 2 * (size_t)NC * 128; }

bool tc_config_fits(const TcPlan* p, const TcConfig& c) {
  if (c.slice < 1 || c.slice > 64 || c.stages < 2 || c.stages > MAX_STAGES) return false;
  const int Bs = std::min(c.slice, p->B);
  return (size_t)c.stages * stage_bytes_of(nc_of(Bs)) + 1024 <= (size_t)p->smem_max;
}

// Assign the items, in list order, each to the CTA that becomes free first, with a cost of its
// chunk count plus a fixed share for its epilogue: the schedule a shared work counter would give,
// made on the host.  Items next to each other in the list then run at about the same time on
// different SMs, so that the data tiles they share are read from HBM about once, and the longest
// CTA finishes close to the mean.  Uploads the items CTA-major and the per-CTA offsets.
static cudaError_t schedule(const std::vector<Item>& items, int grid, Item* d_items, int* d_sched) {
  constexpr long long kEpilogueChunks = 2;
  std::priority_queue<std::pair<long long, int>, std::vector<std::pair<long long, int>>, std::greater<>> free_at;
  for (int b = 0; b < grid; ++b) free_at.push({0, b});
  std::vector<std::vector<int>> per(grid);
  for (int w = 0; w < (int)items.size(); ++w) {
    const auto top = free_at.top();
    free_at.pop();
    per[top.second].push_back(w);
    free_at.push({top.first + (items[w].c1 - items[w].c0) + kEpilogueChunks, top.second});
  }
  std::vector<Item> out;
  std::vector<int> start(grid + 1, 0);
  out.reserve(items.size());
  for (int b = 0; b < grid; ++b) {
    start[b] = (int)out.size();
    for (int w : per[b]) out.push_back(items[w]);
  }
  start[grid] = (int)out.size();
  cudaError_t e = cudaMemcpy(d_items, out.data(), out.size() * sizeof(Item), cudaMemcpyHostToDevice);
  return e != cudaSuccess ? e : cudaMemcpy(d_sched, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice);
}

cudaError_t tc_configure(TcPlan* p, const TcConfig& c) {
  if (!tc_config_fits(p, c)) return cudaErrorInvalidValue;
  cudaError_t e;
  const int Bs = std::min(c.slice, p->B), nS = (p->B + Bs - 1) / Bs, NC = nc_of(Bs);
  const size_t xslice = (size_t)std::max(p->xtiles_inv, p->xtiles_fwd) * (p->bf16 ? 2 : 1) * NC * 128;
  if (xslice * nS != p->xbytes || !p->X) {
    if (p->X) {
      cudaFree(p->X);
      p->bytes -= p->xbytes;
      p->X = nullptr;
    }
    if ((e = tc_alloc((void**)&p->X, xslice * nS, &p->bytes)) != cudaSuccess) return e;
    p->xbytes = xslice * nS;
  }
  p->Bs = Bs;
  p->nS = nS;
  p->NC = NC;
  p->xslice = xslice;
  // Work order (the schedule then hands the items out in this order).  Grouped: the row blocks of
  // each group of 4 consecutive m run together, so that their data tiles are read from HBM about
  // once and the output rows of neighbouring m meet in L2.  Longest first: the classic order for
  // balance.  Order 0 (the default) is grouped in both directions.
  auto grouped = [](const Item& x, const Item& y) {
    if (x.m / 4 != y.m / 4) return x.m / 4 < y.m / 4;
    if (x.i != y.i) return x.i > y.i;
    return x.m < y.m;
  };
  auto longest_first = [](const Item& x, const Item& y) { return (x.c1 - x.c0) > (y.c1 - y.c0); };
  std::vector<Item> inv = p->inv_h, fwd = p->fwd_h;
  if (c.inv_order == 0) std::stable_sort(inv.begin(), inv.end(), grouped);
  else std::stable_sort(inv.begin(), inv.end(), longest_first);
  if (c.fwd_order == 0) std::stable_sort(fwd.begin(), fwd.end(), grouped);
  else std::stable_sort(fwd.begin(), fwd.end(), longest_first);
  if ((e = schedule(inv, p->grid_inv, p->items_inv, p->sched_inv)) != cudaSuccess) return e;
  if ((e = schedule(fwd, p->grid_fwd, p->items_fwd, p->sched_fwd)) != cudaSuccess) return e;
  p->smem = (size_t)c.stages * stage_bytes_of(NC) + 1024;
  p->cfg = c;
  return cudaSuccess;
}

TcConfig tc_config(const TcPlan* p) { return p->cfg; }

cudaError_t tc_setup(TcPlan** out, int L, int s, int B, int bf16, int device) {
  *out = nullptr;
  if (B < 1) return cudaErrorInvalidValue;
  TcPlan* p = new TcPlan();
  size_t ga = 0;
  p->bf16 = bf16 != 0;
  p->L = L;
  p->s = s;
  p->B = B;
  p->nC = (L + TK - 1) / TK;
  p->nI = (L + TM - 1) / TM;
  const int as = s < 0 ? -s : s;
  std::vector<Item>& inv = p->inv_h;
  std::vector<Item>& fwd = p->fwd_h;
  std::vector<long long> xoff(L), abase(L), ibase((size_t)L * std::max(1, (L + TM - 1) / TM), 0);
  std::vector<int> xc0(L);
  long long at = 0, ft = 0, xt = 0;
  for (int m = 0; m < L; ++m) {
    const int lmin = std::max(m, as), im = m / TM;
    xc0[m] = lmin / TK;
    xoff[m] = xt;
    xt += p->nC - xc0[m];
    abase[m] = ft;
    for (int i = im; i < p->nI; ++i) {
      // forward: rows l in block i with l >= m (rows l < |s| come out as zeros), K = m' <= l
      fwd.push_back({m, i, 0, std::min(p->nC, 4 * i + 4), ft});
      ft += 4 * i + 4;
    }
    for (int i = 0; i < p->nI; ++i) {
      // inverse: rows m' in block i, K = l >= max(m, m', |s|)
      const int c0 = std::max(lmin / TK, (i * TM) / TK);
      if (c0 < p->nC) {
        ibase[(size_t)m * p->nI + i] = at - c0;
        inv.push_back({m, i, c0, p->nC, at});
        at += p->nC - c0;
      }
    }
  }
  p->n_inv = (int)inv.size();
  p->n_fwd = (int)fwd.size();
  p->tiles_A = ft;
  p->tiles_inv = at;
  p->xtiles_inv = xt;
  p->xtiles_fwd = (long long)L * p->nC;
  cudaError_t e;
  {
    int sms = 0, optin = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) goto fail;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess) goto fail;
    p->grid = sms;
    p->smem_max = optin - 2048;  // the kernel's static shared memory and alignment slack
  }
  // the inverse leaves one SM to the recursion that writes the forward's operands meanwhile
  p->grid_inv = std::max(1, std::min(p->grid - 1, (int)inv.size()));
  p->grid_fwd = std::max(1, std::min(p->grid, (int)fwd.size()));
  if ((e = tc_alloc((void**)&p->items_inv, inv.size() * sizeof(Item), &p->bytes)) != cudaSuccess) goto fail;
  if ((e = tc_alloc((void**)&p->items_fwd, fwd.size() * sizeof(Item), &p->bytes)) != cudaSuccess) goto fail;
  if ((e = tc_alloc((void**)&p->sched_inv, (p->grid_inv + 1) * sizeof(int), &p->bytes)) != cudaSuccess) goto fail;
  if ((e = tc_alloc((void**)&p->sched_fwd, (p->grid_fwd + 1) * sizeof(int), &p->bytes)) != cudaSuccess) goto fail;
  ga = (size_t)(p->bf16 ? 2 : 1) * A_PART;  // bytes of an A tile in global memory
  if ((e = tc_alloc((void**)&p->A, (size_t)ft * ga, &p->bytes)) != cudaSuccess) goto fail;
  // zero once (entries no call writes stay zero); cudaMemset is asynchronous on the legacy
  // stream, and the plans' packing and recursions run on non-blocking streams: wait for it
  if ((e = cudaMemset(p->A, 0, (size_t)ft * ga)) != cudaSuccess) goto fail;
  if ((e = tc_alloc((void**)&p->A_inv, (size_t)at * ga, &p->bytes)) != cudaSuccess) goto fail;
  if ((e = cudaMemset(p->A_inv, 0, (size_t)at * ga)) != cudaSuccess) goto fail;
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) goto fail;
  if ((e = tc_alloc((void**)&p->ibase, ibase.size() * sizeof(long long), &p->bytes)) != cudaSuccess) goto fail;
  if ((e = cudaMemcpy(p->ibase, ibase.data(), ibase.size() * sizeof(long long), cudaMemcpyHostToDevice)) != cudaSuccess)
    goto fail;
  if ((e = tc_alloc((void**)&p->abase, L * sizeof(long long), &p->bytes)) != cudaSuccess) goto fail;
  if ((e = tc_alloc((void**)&p->xoff, L * sizeof(long long), &p->bytes)) != cudaSuccess) goto fail;
  if ((e = tc_alloc((void**)&p->xc0, L * sizeof(int), &p->bytes)) != cudaSuccess) goto fail;
  if ((e = cudaMemcpy(p->abase, abase.data(), L * sizeof(long long), cudaMemcpyHostToDevice)) != cudaSuccess) goto fail;
  if ((e = cudaMemcpy(p->xoff, xoff.data(), L * sizeof(long long), cudaMemcpyHostToDevice)) != cudaSuccess) goto fail;
  if ((e = cudaMemcpy(p->xc0, xc0.data(), L * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) goto fail;
  {
    // Function attributes are process-wide upper bounds: the device's limit, so that plans of
    // every configuration can launch with their own amounts.
    if ((e = prefer_shared(pack_a_kernel<true, true>)) != cudaSuccess || (e = prefer_shared(pack_a_kernel<true, false>)) != cudaSuccess ||
        (e = prefer_shared(pack_a_kernel<false, true>)) != cudaSuccess || (e = prefer_shared(pack_a_kernel<false, false>)) != cudaSuccess)
      goto fail;
    if (p->bf16) {
      if ((e = gemm_attrs(tc_gemm_kernel<false, true>, p->smem_max)) != cudaSuccess) goto fail;
      if ((e = gemm_attrs(tc_gemm_kernel<true, true>, p->smem_max)) != cudaSuccess) goto fail;
      if ((e = prefer_shared(pack_v_kernel<true>)) != cudaSuccess) goto fail;
    } else {
      if ((e = gemm_attrs(tc_gemm_kernel<false, false>, p->smem_max)) != cudaSuccess) goto fail;
      if ((e = gemm_attrs(tc_gemm_kernel<true, false>, p->smem_max)) != cudaSuccess) goto fail;
      if ((e = prefer_shared(pack_v_kernel<false>)) != cudaSuccess) goto fail;
    }
  }
  if ((e = tc_configure(p, TcConfig())) != cudaSuccess) goto fail;
  *out = p;
  return cudaSuccess;
fail:
  tc_destroy(p);
  return e;
}

void tc_destroy(TcPlan* p) {
  if (!p) return;
  void* ptrs[] = {p->items_inv, p->items_fwd, p->sched_inv, p->sched_fwd, p->A, p->A_inv, p->abase, p->ibase, p->X, p->xoff, p->xc0};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete p;
}

size_t tc_bytes(const TcPlan* p) { return p ? p->bytes : 0; }

InvTiles tc_inverse_tiles(const TcPlan* p) {
  InvTiles t;
  if (p && !p->bf16) {
    t.A = p->A_inv;
    t.ibase = p->ibase;
    t.nI = p->nI;
    t.nC = p->nC;
    t.ntiles = p->tiles_inv;
  }
  return t;
}

ATiles tc_a_tiles(const TcPlan* p) {
  ATiles t;
  if (p && !p->bf16) {
    t.A = p->A;
    t.abase = p->abase;
    t.ntiles = p->tiles_A;
  }
  return t;
}

cudaError_t tc_pack_a(TcPlan* p, int forward, const double* table, const float* U, cudaStream_t st, int* launches) {
  // one block per (item, chunk): grid.x covers the longest item (at most nC chunks), grid.y the items
  const dim3 gf(p->nC, p->n_fwd), gi(p->nC, p->n_inv);
  if (forward && p->bf16)
    pack_a_kernel<true, true><<<gf, 256, 0, st>>>(p->L, p->s, p->items_fwd, table, U, p->A, p->tiles_A);
  else if (forward)
    pack_a_kernel<true, false><<<gf, 256, 0, st>>>(p->L, p->s, p->items_fwd, table, U, p->A, p->tiles_A);
  else if (p->bf16)
    pack_a_kernel<false, true><<<gi, 256, 0, st>>>(p->L, p->s, p->items_inv, table, U, p->A_inv, p->tiles_inv);
  else
    pack_a_kernel<false, false><<<gi, 256, 0, st>>>(p->L, p->s, p->items_inv, table, U, p->A_inv, p->tiles_inv);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t tc_pack_data(TcPlan* p, const void* src, cudaStream_t st, int* launches) {
  const dim3 g(p->nC, (p->L + 15) / 16, p->nS);
  if (p->bf16)
    pack_v_kernel<true><<<g, 256, 0, st>>>(p->L, p->s, p->B, p->Bs, p->xslice, p->NC, p->xc0, p->xoff,
                                           (const float2*)src, p->X);
  else
    pack_v_kernel<false><<<g, 256, 0, st>>>(p->L, p->s, p->B, p->Bs, p->xslice, p->NC, p->xc0, p->xoff,
                                            (const float2*)src, p->X);
  *launches += 1;
  return cudaGetLastError();
}

TileOut tc_forward_tiles(const TcPlan* p) {
  TileOut o;
  o.X = p->X;
  o.NC = p->NC;
  o.nC = p->nC;
  o.mode = p->bf16 ? 2 : 1;
  o.Bs = p->Bs;
  o.xslice = p->xslice;
  o.xbytes = p->xbytes;
  return o;
}

cudaError_t tc_gemm(TcPlan* p, int forward, void* out, const void* ph, int* status, long long wait_ns, cudaStream_t st,
                    int* launches) {
  // one launch per slice of fields; every slice reads the same A tiles
  for (int sl = 0; sl < p->nS; ++sl) {
    TcArgs a;
    a.L = p->L;
    a.s = p->s;
    a.B = std::min(p->Bs, p->B - sl * p->Bs);
    a.NC = p->NC;
    a.stages = p->cfg.stages;
    a.sched = forward ? p->sched_fwd : p->sched_inv;
    a.items = forward ? p->items_fwd : p->items_inv;
    a.A = forward ? p->A : p->A_inv;
    a.X = p->X + (size_t)sl * p->xslice;
    a.xoff = p->xoff;
    a.xc0 = p->xc0;
    a.ph = (const float2*)ph;
    const size_t per_field = forward ? (size_t)p->L * p->L : (size_t)(2 * p->L - 1) * p->L;
    a.out = (float2*)out + (size_t)sl * p->Bs * per_field;
    a.status = status;
    a.wait_ns = wait_ns;
    a.a_tiles = forward ? p->tiles_A : p->tiles_inv;
    a.x_tiles = (long long)(p->xslice / ((p->bf16 ? 2 : 1) * (size_t)p->NC * 128));
    a.out_n = (long long)a.B * (long long)per_field;
    const int grid = forward ? p->grid_fwd : p->grid_inv;
    if (forward && p->bf16)
      tc_gemm_kernel<true, true><<<grid, THREADS, p->smem, st>>>(a);
    else if (forward)
      tc_gemm_kernel<true, false><<<grid, THREADS, p->smem, st>>>(a);
    else if (p->bf16)
      tc_gemm_kernel<false, true><<<grid, THREADS, p->smem, st>>>(a);
    else
      tc_gemm_kernel<false, false><<<grid, THREADS, p->smem, st>>>(a);
    *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

SSHT_BOUNDS_TU(contract_tc)

}  // namespace ssht
