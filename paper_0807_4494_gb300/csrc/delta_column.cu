// Delta^l = d^l(pi/2) for l = 0 .. L-1, FP64, one column m at a time by the three-term relation
// in the first index m' -- the default way the plans make the table (the Risbo recursion of
// Sec. 2.2, which the paper uses, is in delta.cu and selected by SSHT_FLAG_RISBO).
//
// The relation.  d^l(pi/2) rotates the z axis onto the x axis, so it turns J_z into J_x:
// J_x Delta^l = Delta^l J_z with the ladder elements <m'+-1| J_+- |m'> = sqrt((l -+ m')(l +- m' + 1)).
// Written out for row m' and column m of degree l:
//   sqrt((l-m'+1)(l+m')) Delta_{m'-1,m} + sqrt((l-m')(l+m'+1)) Delta_{m'+1,m} = 2m Delta_{m'm},
// i.e. Delta_{m'-1,m} = 2m a(m') Delta_{m'm} - b(m') Delta_{m'+1,m} with
//   a(m') = 1/sqrt((l-m'+1)(l+m')),  b(m') = sqrt((l-m')(l+m'+1)) a(m')   (b(l) = 0).
// It starts from the first row, which eqn wignerd_b gives in closed form at beta = pi/2:
//   Delta_{l m} = (-1)^{l-m} 2^{-l} sqrt(C(2l, l+m)) = (-1)^{l-m} 2^{-l} prod_{k=m+1}^{l} g(k),
//   g(k) = sqrt((l+k)/(l-k+1)).
// Run downwards in m' (from the first row into the interior) the relation moves from the
// region where d(pi/2) decays towards the one where it oscillates, the stable direction; the
// table matches the oracle's Risbo recursion to ~1e-14 up to l = 2047.
//
// Work.  Every degree is independent once its first row is known, so there is no hand-off
// between CTAs: a task is one degree l and one block of 32 columns m = 32b + lane, a warp walks
// m' from l down to 32b (the octant part m' >= m of its columns, plus the 32 x 32 diagonal
// block), writing row m' of its columns directly (coalesced) and the transposed entries
// Delta_{m m'} = (-1)^{m'-m} Delta_{m'm} of rows m through a 32 x 32 shared-memory block (again
// coalesced).  Each update is 2 FP64 instructions, b(m') Delta_{m'+1,m} and the fused
// multiply-add (the FP64 pipe is the scarce one on this part: 2 lanes per SM and clock); the
// coefficient 2m a(m') is the exactly rounded product made on the integer pipe (int_mul.h), and
// the a(m'), b(m') of 32 consecutive m' are made once per chunk by the warp from the sqrt tables.
// Tasks are taken longest first from an atomic counter.
//
// Range.  Delta_{l,l} = 2^{-l} is below the FP64 normal range for l > 1022.  For band-limits
// above 1024 each lane carries its own binary exponent E (true value = stored * 2^E) until the
// value is back in range; entries below 2^-1021 are written as 0 (they are below 1e-307 and
// contribute nothing to any transform).
#include "ssht_internal.h"
#include "bounds.cuh"
#include "f32_round.h"
#include "int_mul.h"
#include "tc_common.cuh"

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <vector>

namespace ssht {
namespace {

__device__ __forceinline__ size_t delta_offset_dev(long long l) { return (size_t)(l * (l + 1) * (2 * l + 1) / 6); }

constexpr int kColWarps = 8;
constexpr int kColThreads = 32 * kColWarps;
constexpr int kStageDoubles = 32 * 33;              // a warp's transposition block (padded rows)
constexpr int kWarpDoubles = kStageDoubles + 64;    // + the chunk's coefficients (a, b or alpha, p)
constexpr size_t kColSmem = (size_t)kColWarps * kWarpDoubles * sizeof(double);

struct ColumnParams {
  int L;
  int ntasks;
  const int2* tasks;       // (l, b), longest first
  const double* sq;        // sqrt(k), k < 2L + 4
  const double* rsq;       // 1/sqrt(k), k >= 1
  double* table;           // quadrant table, entry (l, m', m) at offset(l) + m'(l+1) + m
  unsigned int* counter;   // next task (zeroed before the launch)
  // tile output (3xTF32 plans): A_m[l][m'] = Uf_l[m'] Delta^l_{m'm} into the forward tile layout
  const float* Uf;         // U_l[m'] in FP32 at l(l+1)/2 + m'
  const double* alc;       // alpha(l, m') of the rescaled relation at l(l+1)/2 + m'
  const float* pc;         // p(l, m') at l(l+1)/2 + m'
  uint8_t* A;              // tiles (m, l / 128, m' / 32) of 128 rows l x 32 K values m' (FP32)
  const long long* ab2;    // per M: index of the tile (M, M / 128, 0) less 2 (M/128) (M/128 + 1)
  long long extent;        // entries of the table, or tiles of A (index checks)
};

// Writes A_M[l][K] = x (FP32) into row l mod 128 of tile (M, l / 128, K / 32): the 3xTF32 tiles
// hold one FP32 part in global memory (the contraction splits it into hi + lo on arrival).
__device__ __forceinline__ void put_a(uint8_t* A, long long tile, long long ntiles, int site, int row, int k, float x) {
  if (!in_bounds(tile, ntiles, site)) return;
  uint8_t* t = A + (size_t)tile * tc::kAPart;
  *(float*)(t + tc::sw128(row, 4 * k)) = x;
}
// The same with the swizzled offset of (row, K) in the tile already made.
__device__ __forceinline__ void put_a_at(uint8_t* A, long long tile, long long ntiles, int site, uint32_t off, float x) {
  if (!in_bounds(tile, ntiles, site)) return;
  *(float*)(A + (size_t)tile * tc::kAPart + off) = x;
}

__device__ __forceinline__ double flip_sign(double v, bool neg) {
  return __hiloint2double(__double2hiint(v) ^ (neg ? (int)0x80000000 : 0), __double2loint(v));
}
// Unbiased binary exponent of a normal nonzero double, and the same mantissa with exponent e
// (integer operations on the bit pattern; no FP64 instruction).
__device__ __forceinline__ int exp_of(double v) { return ((__double2hiint(v) >> 20) & 0x7ff) - 1023; }
__device__ __forceinline__ double with_exp(double v, int e) {
  const int hi = (__double2hiint(v) & (int)0x800fffff) | ((e + 1023) << 20);
  return __hiloint2double(hi, __double2loint(v));
}

// First row of degree l for the 32 columns m = m0 + lane (the whole warp calls it, m0 a multiple of
// 32): Delta_{l m} = (-1)^{l-m} v 2^{*ge - l} with v in [1, 2^194) returned, from
// prod_{k=m+1}^{l} g(k), g(k) = sqrt((l+k)/(l-k+1)) >= 1.
__device__ __forceinline__ double first_row(int l, int m0, int lane, const double* __restrict__ sq,
                                            const double* __restrict__ rsq, int* ge_out) {
  const int m = m0 + lane;
  // G = prod_{k = m0+33}^{l} g(k) as gm * 2^ge: each lane multiplies every 32nd factor (at most
  // 64 factors of at most sqrt(2l) <= 64, so no overflow), then the warp multiplies the lanes'
  // products with their exponents split off (the whole product reaches 2^l).
  double gm = 1.0;
  for (int k = m0 + 33 + lane; k <= l; k += 32) gm = __dmul_rn(gm, __dmul_rn(sq[l + k], rsq[l - k + 1]));
  int ge = exp_of(gm);
  gm = with_exp(gm, 0);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const double om = __shfl_xor_sync(0xffffffffu, gm, d);
    const int oe = __shfl_xor_sync(0xffffffffu, ge, d);
    gm = __dmul_rn(gm, om);  // in [1, 4)
    ge += oe + exp_of(gm);
    gm = with_exp(gm, 0);
  }
  // h = prod_{k = m+1}^{min(m0+32, l)} g(k): suffix product of the lanes' own factors g(m+1)
  // (at most 32 factors, at most 2^192).
  double h = (m + 1 <= l) ? __dmul_rn(sq[l + m + 1], rsq[l - m]) : 1.0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double o = __shfl_down_sync(0xffffffffu, h, d);
    if (lane + d < 32) h = __dmul_rn(h, o);
  }
  *ge_out = ge;
  return __dmul_rn(h, gm);
}

// Folds the exponent of the scaled variant back in, or moves the values away from overflow.
__device__ __forceinline__ void rescale_exponent(double& cur, double& prev, int& E) {
  const int x = exp_of(cur);
  if (x + E >= -1021) {  // back in the normal range
    cur = ldexp(cur, E);
    prev = ldexp(prev, E);
    E = 0;
  } else if (x > 512) {
    cur = __dmul_rn(cur, 0x1p-512);
    prev = __dmul_rn(prev, 0x1p-512);
    E += 512;
  }
}

template <bool SCALED>
__global__ void __launch_bounds__(kColThreads, 2) column_recursion_kernel(ColumnParams P) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* stage = smem + warp * kWarpDoubles;
  double* coef = stage + kStageDoubles;  // a(m') of the chunk, then b(m')
  const double* __restrict__ sq = P.sq;
  const double* __restrict__ rsq = P.rsq;
  for (;;) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(P.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= P.ntasks) break;
    const int2 task = P.tasks[t];
    const int l = task.x, m0 = 32 * task.y, m = m0 + lane;
    const bool act = m <= l;

    // ---- first row: Delta_{l m} = (-1)^{l-m} v 2^{ge - l} ----
    int ge;
    const double v = first_row(l, m0, lane, sq, rsq, &ge);
    int E = 0;                          // SCALED: true value = stored * 2^E (E < 0 while out of range)
    double cur;
    if (!act) {
      cur = 0.0;
    } else if (!SCALED || exp_of(v) + ge - l >= -1021) {
      cur = flip_sign(ldexp(v, ge - l), ((l - m) & 1) != 0);
    } else {
      cur = flip_sign(v, ((l - m) & 1) != 0);
      E = ge - l;
    }
    double prev = 0.0;
    double* __restrict__ T = P.table + delta_offset_dev(l);
    const size_t row = (size_t)l + 1;

    // ---- rows m' = l .. m0 ----
    for (int mp = l; mp >= m0; --mp) {
      const int j = mp & 31;
      if (mp == l || j == 31) {
        // coefficients a(m'), b(m') of the chunk of m' in [mp & ~31, (mp & ~31) + 31]
        __syncwarp();
        const int k = (mp & ~31) + lane;
        double a = 0.0, b = 0.0;
        if (k >= 1 && k <= l) {
          a = __dmul_rn(rsq[l - k + 1], rsq[l + k]);
          b = __dmul_rn(__dmul_rn(sq[l - k], sq[l + k + 1]), a);
        }
        coef[lane] = a;
        coef[32 + lane] = b;
        __syncwarp();
      }
      const double out = (SCALED && E != 0) ? 0.0 : cur;
      if (act && in_bounds((long long)delta_offset_dev(l) + (long long)(mp * row + m), P.extent, kbColumnTable))
        T[(size_t)mp * row + m] = out;
      if (mp >= m0 + 32) {
        // transposed entry Delta_{m m'} = (-1)^{m'-m} Delta_{m'm}, written a 32-column chunk at a time
        stage[lane * 33 + j] = flip_sign(out, ((mp - m) & 1) != 0);
        if (j == 0) {
          __syncwarp();
          const int c = mp + lane;
          for (int r = 0; r < 32 && m0 + r <= l; ++r)
            if (c <= l && in_bounds((long long)delta_offset_dev(l) + (long long)((m0 + r) * row + c), P.extent,
                                    kbColumnTable))
              T[(size_t)(m0 + r) * row + c] = stage[r * 33 + lane];
          __syncwarp();
        }
      }
      if (mp > m0) {
        const double c = mul_small_rn(coef[j], (uint32_t)m, 1);  // 2m a(m'), on the integer pipe
        const double nxt = __fma_rn(c, cur, -__dmul_rn(coef[32 + j], prev));
        prev = cur;
        cur = nxt;
        if (SCALED && E != 0) {
          const int x = exp_of(cur);
          if (x + E >= -1021) {  // back in the normal range: fold the exponent in
            cur = ldexp(cur, E);
            prev = ldexp(prev, E);
            E = 0;
          } else if (x > 512) {  // keep the stored values far from overflow
            cur = __dmul_rn(cur, 0x1p-512);
            prev = __dmul_rn(prev, 0x1p-512);
            E += 512;
          }
        }
      }
    }
  }
}

// The same walk writing the A tiles of a 3xTF32 plan instead of the table.  With x = Delta_{m'm}
// in lane m at step m' (row), the entry serves two tiles: A_{m'}[l][m] = U_l[m] (-1)^{m'-m} x, a
// row of 32 consecutive K values across the warp (written at once), for every row m' >= 32b; and
// A_m[l][m'] = U_l[m'] x, which goes through the transposition block like the table's transposed
// entries, for m' >= 32b + 32 -- together every (M, K) pair of the degree once.  Every write of a
// task lands on row l mod 128, K = lane of its tile, one swizzled offset; the tile of column group
// M is ab2[M] + 2 il (il + 1) + chunk (ab2 holds the plan's per-M tile base less the row blocks
// below M's own).
//
// The tiles need Delta only in FP32, so here the relation runs rescaled: with
// Delta_{m'm} = p(l, m') y_{m'}, p(l, l) = p(l, l-1) = 1 and p(l, m'-1) = b(m') p(l, m'+1), it reads
//   y_{m'-1} = m alpha(l, m') y_{m'} - y_{m'+1},   alpha(l, m') = 2 a(m') p(l, m') / p(l, m'-1),
// one FP64 fused multiply-add an update (the coefficient m alpha is the integer-pipe product).  p
// lies in [0.15, 1] up to l = 2047 and multiplies the FP32 output; alpha and p are plan-time
// tables (rescale_tables_kernel).  Each value is rounded to FP32 once and staged as FP32, so a
// CTA needs half the table kernel's shared memory and three fit an SM.
// The forward's tiles are needed only after the inverse's and the forward's torus passes, so the
// persistent grid takes one CTA an SM and runs beside those passes, which keep two of their three
// CTAs an SM (GB300, L = 1024, B = 64: 12.09 ms a step, against 12.11 with two CTAs an SM and 12.15
// with three).
#ifndef SSHT_COLUMN_CTAS
#define SSHT_COLUMN_CTAS 1
#endif
constexpr int kTileStageFloats = 32 * 33;
constexpr int kTileWarpBytes = kTileStageFloats * 4 + 32 * 8 + 32 * 4;  // stage, alpha[32], p[32]
constexpr size_t kTileSmem = (size_t)kColWarps * kTileWarpBytes;

template <bool SCALED>
__global__ void __launch_bounds__(kColThreads, 3) column_tiles_kernel(ColumnParams P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* stage = reinterpret_cast<float*>(smraw + warp * kTileWarpBytes);
  double* alw = reinterpret_cast<double*>(smraw + warp * kTileWarpBytes + kTileStageFloats * 4);
  float* pw = reinterpret_cast<float*>(alw + 32);
  const double* __restrict__ sq = P.sq;
  const double* __restrict__ rsq = P.rsq;
  const long long ntri = (long long)P.L * (P.L + 1) / 2;
  for (;;) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(P.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= P.ntasks) break;
    const int2 task = P.tasks[t];
    const int l = task.x, m0 = 32 * task.y, m = m0 + lane;
    const bool act = m <= l;

    // ---- first row: y_l = Delta_{l m} = (-1)^{l-m} v 2^{ge - l} (p(l, l) = 1) ----
    int ge;
    const double v = first_row(l, m0, lane, sq, rsq, &ge);
    int E = 0;
    double cur;
    if (!act) {
      cur = 0.0;
    } else if (!SCALED || exp_of(v) + ge - l >= -1021) {
      cur = flip_sign(ldexp(v, ge - l), ((l - m) & 1) != 0);
    } else {
      cur = flip_sign(v, ((l - m) & 1) != 0);
      E = ge - l;
    }
    double prev = 0.0;
    const int il = l >> 7;
    const long long ilpre = 2ll * il * (il + 1);
    const long long tadd = ilpre + (m0 >> 5);
    const uint32_t off = tc::sw128(l & 127, 4 * lane);
    const size_t lrow = (size_t)l * (l + 1) / 2;  // row l of the degree-major tables
    const double md = (double)m;
    // U_l[m] of this lane's column and the tile base of its row M = m (the transposed writes)
    float u_lane = 0.f;
    long long base_lane = 0;
    if (act) {
      u_lane = __ldg(&P.Uf[lrow + m]);
      base_lane = __ldg(&P.ab2[m]) + ilpre;
    }
    // the base of row M = m' (a load), fetched one step ahead
    long long ab_cur = __ldg(&P.ab2[l]), ab_next = 0;
    int mp = l;
    // one row; the coefficient m alpha of its update comes from the FP64 pipe or from the integer
    // pipe (the same exactly rounded product), alternately, so that the two pipes share the work
    auto row = [&](auto on_fp64) {
      if (mp > m0) ab_next = __ldg(&P.ab2[mp - 1]);
      const int j = mp & 31;
      if (mp == l || j == 31) {
        // alpha(l, m') and p(l, m') of the chunk of m' in [mp & ~31, (mp & ~31) + 31]
        __syncwarp();
        const int k = (mp & ~31) + lane;
        double al = 0.0;
        float pk = 0.f;
        if (k <= l && in_bounds((long long)(lrow + k), ntri, kbColumnCoef)) {
          al = __ldg(&P.alc[lrow + k]);
          pk = __ldg(&P.pc[lrow + k]);
        }
        alw[lane] = al;
        pw[lane] = pk;
        __syncwarp();
      }
      const float x = f64_to_f32_rn((SCALED && E != 0) ? 0.0 : cur);  // y_{m'} in FP32
      if (act) put_a_at(P.A, ab_cur + tadd, P.extent, kbColumnTile, off, (u_lane * pw[j]) * (((mp - m) & 1) ? -x : x));
      if (mp >= m0 + 32) {
        stage[lane * 33 + j] = x;
        if (j == 0) {
          // A_M[l][m'] for the columns M = m0 + r, m' = mp + lane: U_l[m'] p(l, m') y
          __syncwarp();
          const int c = mp + lane;
          const float uc = c <= l ? __ldg(&P.Uf[lrow + c]) * __ldg(&P.pc[lrow + c]) : 0.f;
          const int cb = mp >> 5;
          for (int r = 0; r < 32 && m0 + r <= l; ++r) {
            const long long tile = __shfl_sync(0xffffffffu, base_lane, r) + cb;
            if (c <= l) put_a_at(P.A, tile, P.extent, kbColumnTile, off, uc * stage[r * 33 + lane]);
          }
          __syncwarp();
        }
      }
      if (mp > m0) {
        double c;
        if constexpr (decltype(on_fp64)::value)
          c = __dmul_rn(md, alw[j]);
        else
          c = mul_small_rn(alw[j], (uint32_t)m, 0);
        const double nxt = __fma_rn(c, cur, -prev);
        prev = cur;
        cur = nxt;
        if (SCALED && E != 0) rescale_exponent(cur, prev, E);
      }
      ab_cur = ab_next;
      --mp;
    };
    for (;;) {
      row(std::true_type{});
      if (mp < m0) break;
      row(std::false_type{});
      if (mp < m0) break;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// One lane per degree: the inverse contraction's A tiles (rows m', K = l), 3xTF32 plans.
//
// The inverse's tile rows run along K = l, so here a warp takes 32 consecutive degrees
// l = 32 kc + lane and one column m and walks m' from the top degree down to m, lane l starting
// at m' = l from its first-row entry.  At step m' the lanes hold Delta^l_{m'm} for 32 consecutive
// l: A_m[m'][l] = U_l[m'] Delta^l_{m'm} is one 32-wide tile row, and so (for m' > m) is
// A_{m'}[m][l] = U_l[m] (-1)^{m'-m} Delta^l_{m'm} -- every entry of A with m' >= m from the first
// write, with m' < m from the second, each once.  The relation runs rescaled as in the column
// recursion's tile output (Delta = p y, y_{m'-1} = m alpha y_{m'} - y_{m'+1}: one FP64 instruction
// an update); alpha(l, m') and p(l, m') differ per lane here, so they, the first rows and the
// transposed U come from plan-time tables in the triangle layout [r][l], l >= r, read 32
// consecutive l at a time.  The index of (r, l) in that layout drops by L - r when r drops by one,
// and the tile base of row r by nI, so a step moves both by an addition.
// ---------------------------------------------------------------------------------------------

// Index of (r, l), 0 <= r <= l < L, in the triangle layout [r][l].
__host__ __device__ __forceinline__ size_t tri_idx(long long r, long long l, long long L) {
  return (size_t)(r * L - r * (r - 1) / 2 + (l - r));
}

struct LaneParams {
  int L, as, nI, ntasks;
  const int2* tasks;        // (m, kc), longest first
  const double* alpha;      // alpha(l, m') at tri_idx(m', l)
  const float* p;           // p(l, m') at tri_idx(m', l)
  const double* t1m;        // first rows: Delta_{l m} = t1m 2^t1e at tri_idx(m, l) (t1e = 0 where a
                            // double holds the value)
  const int* t1e;
  const float* ufT;         // U_l[m'] at tri_idx(m', l)
  uint8_t* A;               // inverse tiles (m, m' / 128, l / 32)
  const long long* ibase;   // [m * nI + i]: index of the tile of chunk kc is ibase + kc
  unsigned int* counter;
  long long ntiles;         // tiles of A (index checks)
};

// Resident CTAs an SM of the persistent grid: all four that fit (with one or two the recursion,
// started beside the forward's torus passes, slowed them more than it gained: 12.14 and 12.11 ms
// a step against 11.995 at L = 1024, B = 64).
#ifndef SSHT_LANE_CTAS
#define SSHT_LANE_CTAS 4
#endif

// Rows top .. max(m, 32 kc) are the start-up phase: lane l joins at m' = l from its first-row
// entry.  Below 32 kc every lane of a degree that exists runs, m' < l, and the steady loop needs
// none of the start-up tests.
template <bool SCALED>
__global__ void __launch_bounds__(kColThreads, 4) lane_recursion_kernel(LaneParams P) {
  const int lane = threadIdx.x & 31;
  const int L = P.L;
  const int ntri = L * (L + 1) / 2;
  for (;;) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(P.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= P.ntasks) break;
    const int2 task = P.tasks[t];
    const int m = task.x, kc = task.y;
    const int l = 32 * kc + lane;
    const int top = min(32 * kc + 31, L - 1);
    const int lo = max(m, 32 * kc);
    const bool inl = l < L && l >= m;     // degree l exists and has column m
    const bool wr = inl && l >= P.as;     // U_l vanishes below |s|: those entries stay zero
    const float um = wr ? __ldg(&P.ufT[tri_idx(m, l, L)]) : 0.f;
    const long long* ib_m = P.ibase + (size_t)m * P.nI;
    const uint32_t off_m = tc::sw128(m & 127, 4 * lane);  // (row m, K = l) in the tiles A_{m'}[m][.]
    uint8_t* const A = P.A;
    double cur = 0.0, prev = 0.0;
    int E = 0;
    // the per-row loads (alpha, p, U, tile base) are issued one step ahead, so that their latency
    // overlaps the step before; kidx and ibr follow the row r by additions
    int kidx = top * L - top * (top - 1) / 2 + (l - top);  // tri_idx(top, l)
    const long long* ibr = P.ibase + (size_t)top * P.nI + (m >> 7);
    double ca = 0.0;
    float cp = 0.f, cu = 0.f;
    if (inl && top <= l && in_bounds(kidx, ntri, kbLaneTable)) {
      ca = __ldg(&P.alpha[kidx]);
      cp = __ldg(&P.p[kidx]);
      cu = __ldg(&P.ufT[kidx]);
    }
    long long ct = __ldg(ibr), tb = 0;
    int mp = top;
    // ---- start-up rows top .. lo ----
    for (; mp >= lo; --mp) {
      double na = 0.0;
      float np = 0.f, nu = 0.f;
      long long nt = 0;
      if (mp > m) {
        kidx -= L - mp;
        ibr -= P.nI;
        if (inl && mp - 1 <= l && in_bounds(kidx, ntri, kbLaneTable)) {
          na = __ldg(&P.alpha[kidx]);
          np = __ldg(&P.p[kidx]);
          nu = __ldg(&P.ufT[kidx]);
        }
        nt = __ldg(ibr);
      }
      if (mp == top || (mp & 127) == 127) tb = __ldg(&ib_m[mp >> 7]) + kc;  // tile of row m' of column m
      if (mp == l && inl) {
        const size_t k = tri_idx(m, l, L);
        cur = __ldg(&P.t1m[k]);  // y_l = Delta_{l m} (p(l, l) = 1), or its mantissa with E apart
        E = SCALED ? __ldg(&P.t1e[k]) : 0;
        prev = 0.0;
      }
      if (inl && mp <= l) {
        if (wr) {
          const float x = f64_to_f32_rn((SCALED && E != 0) ? 0.0 : cur);
          put_a(A, tb, P.ntiles, kbLaneTile, mp & 127, lane, (cu * cp) * x);
          if (mp > m) put_a_at(A, ct + kc, P.ntiles, kbLaneTile, off_m, (um * cp) * (((mp - m) & 1) ? -x : x));
        }
        if (mp > m) {
          const double nxt = __fma_rn(mul_small_rn(ca, (uint32_t)m, 0), cur, -prev);  // m alpha, integer pipe
          prev = cur;
          cur = nxt;
          if (SCALED && E != 0) rescale_exponent(cur, prev, E);
        }
      }
      ca = na;
      cp = np;
      cu = nu;
      ct = nt;
    }
    // ---- steady rows lo - 1 .. m + 1: every lane with inl runs, m' < l ----
    // The coefficient m alpha alternates between the FP64 pipe and the integer pipe (both give
    // the exactly rounded product), which shares the work between the two.
    const double md = (double)m;
    auto steady = [&](auto on_fp64) {
      kidx -= L - mp;
      ibr -= P.nI;
      double na = 0.0;
      float np = 0.f, nu = 0.f;
      if (inl && in_bounds(kidx, ntri, kbLaneTable)) {
        na = __ldg(&P.alpha[kidx]);
        np = __ldg(&P.p[kidx]);
        nu = __ldg(&P.ufT[kidx]);
      }
      const long long nt = __ldg(ibr);
      if ((mp & 127) == 127) tb = __ldg(&ib_m[mp >> 7]) + kc;
      if (inl) {
        if (wr) {
          const float x = f64_to_f32_rn((SCALED && E != 0) ? 0.0 : cur);
          put_a(A, tb, P.ntiles, kbLaneTile, mp & 127, lane, (cu * cp) * x);
          put_a_at(A, ct + kc, P.ntiles, kbLaneTile, off_m, (um * cp) * (((mp - m) & 1) ? -x : x));
        }
        double c;
        if constexpr (decltype(on_fp64)::value)
          c = __dmul_rn(md, ca);
        else
          c = mul_small_rn(ca, (uint32_t)m, 0);
        const double nxt = __fma_rn(c, cur, -prev);
        prev = cur;
        cur = nxt;
        if (SCALED && E != 0) rescale_exponent(cur, prev, E);
      }
      ca = na;
      cp = np;
      cu = nu;
      ct = nt;
      --mp;
    };
    while (mp > m + 1) {
      steady(std::true_type{});
      steady(std::false_type{});
    }
    if (mp > m) steady(std::false_type{});
    // ---- the last row m' = m, if the steady loop reached it ----
    if (m < lo) {
      if ((m & 127) == 127) tb = __ldg(&ib_m[m >> 7]) + kc;
      if (wr) put_a(A, tb, P.ntiles, kbLaneTile, m & 127, lane, (cu * cp) * f64_to_f32_rn((SCALED && E != 0) ? 0.0 : cur));
    }
  }
}

// Plan-time tables of the tile-writing recursions: the first rows (one warp per degree and block
// of 32 columns, the arithmetic of the column recursion), the rescaled relation's alpha(l, m') and
// p(l, m'), and U transposed.
__global__ void lane_first_rows_kernel(int L, const double* __restrict__ sq, const double* __restrict__ rsq,
                                       double* __restrict__ t1m, int* __restrict__ t1e) {
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.y, m0 = 32 * (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)), m = m0 + lane;
  if (m0 > l) return;  // whole warp
  int ge;
  const double v = first_row(l, m0, lane, sq, rsq, &ge);
  if (m <= l) {
    // Delta_{l m} itself where a double holds it (always for L <= 1024: the scaled variant of the
    // recursion runs above that); else the mantissa and the exponent apart
    const size_t k = tri_idx(m, l, L);
    const bool whole = L <= 1024 || exp_of(v) + ge - l >= -1021;
    t1m[k] = flip_sign(whole ? ldexp(v, ge - l) : v, ((l - m) & 1) != 0);
    t1e[k] = whole ? 0 : ge - l;
  }
}

// One thread per degree l walks m' = l .. 0: a(m'), b(m') from the sqrt tables (the products of
// the unscaled relation), p(l, l) = p(l, l-1) = 1, p(l, m'-1) = b(m') p(l, m'+1) and
// alpha(l, m') = 2 a(m') p(l, m') / p(l, m'-1) (alpha(l, 0) is never used: no step leaves m' = 0).
// Written degree-major (l(l+1)/2 + m', the column recursion's chunks) and in the triangle layout
// tri_idx(m', l) (the degree-lane recursion), with U_l[m'] transposed beside them.
__global__ void rescale_tables_kernel(int L, const double* __restrict__ sq, const double* __restrict__ rsq,
                                      const float* __restrict__ Uf, double* __restrict__ alc, float* __restrict__ pc,
                                      double* __restrict__ alT, float* __restrict__ pT, float* __restrict__ ufT) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  const size_t row = (size_t)l * (l + 1) / 2;
  double p_up = 1.0, p_cur = 1.0;  // p(l, m'+1) and p(l, m') at m' = l (the first is not used there)
  for (int mp = l; mp >= 0; --mp) {
    double p_dn = 0.0, al = 0.0;
    if (mp >= 1) {
      const double a = __dmul_rn(rsq[l - mp + 1], rsq[l + mp]);
      const double b = __dmul_rn(__dmul_rn(sq[l - mp], sq[l + mp + 1]), a);
      p_dn = mp == l ? 1.0 : __dmul_rn(b, p_up);
      al = __ddiv_rn(__dmul_rn(2.0 * a, p_cur), p_dn);
    }
    const size_t kt = tri_idx(mp, l, L);
    const float pf = __double2float_rn(p_cur);
    alc[row + mp] = al;
    pc[row + mp] = pf;
    alT[kt] = al;
    pT[kt] = pf;
    ufT[kt] = Uf[row + mp];
    p_up = p_cur;
    p_cur = p_dn;
  }
}

// ab2[M] = abase[M] - 2 i (i + 1), i = M / 128: the tile of (M, row block il, chunk c) of the
// forward layout is ab2[M] + 2 il (il + 1) + c.
__global__ void tile_base_kernel(int L, const long long* __restrict__ abase, long long* __restrict__ ab2) {
  const int M = blockIdx.x * blockDim.x + threadIdx.x;
  if (M >= L) return;
  const long long i = M >> 7;
  ab2[M] = abase[M] - 2 * i * (i + 1);
}

}  // namespace

// Tasks (l, b) for every degree l < L and block b <= l / 32 of 32 columns, longest first (a task
// of degree l and block b walks l - 32b + 1 rows).
static std::vector<int2> column_tasks(int L) {
  std::vector<int2> t;
  for (int l = 0; l < L; ++l)
    for (int b = 0; 32 * b <= l; ++b) t.push_back(make_int2(l, b));
  std::stable_sort(t.begin(), t.end(), [](const int2& x, const int2& y) { return x.x - 32 * x.y > y.x - 32 * y.y; });
  return t;
}

cudaError_t column_setup(DeltaWork& w, int L, int device) {
  cudaError_t e;
  int sms = 0, per_sm = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
  const bool scaled = L > 1024;
  const void* fn = scaled ? (const void*)column_recursion_kernel<true> : (const void*)column_recursion_kernel<false>;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColSmem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared)) !=
      cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kColThreads, kColSmem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const std::vector<int2> tasks = column_tasks(L);
  w.method = kDeltaColumn;
  w.threads = kColThreads;
  w.blocks = sms * std::min(per_sm, 2);
  w.smem = kColSmem;
  w.ntasks = (int)tasks.size();
  if ((e = dev_malloc(&w.table, delta_offset(L) * sizeof(double))) != cudaSuccess) return e;
  if ((e = dev_malloc(&w.sqrt_tab, 2 * (2 * (size_t)L + 4) * sizeof(double))) != cudaSuccess) return e;
  if ((e = dev_malloc(&w.barrier, 4 * sizeof(unsigned int))) != cudaSuccess) return e;
  if ((e = dev_malloc(&w.status, sizeof(int))) != cudaSuccess) return e;
  if ((e = dev_malloc(&w.tasks, tasks.size() * sizeof(int2))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(w.tasks, tasks.data(), tasks.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if ((e = cudaMemset(w.status, 0, sizeof(int))) != cudaSuccess) return e;
  w.bytes = (delta_offset(L) + 2 * (2 * (size_t)L + 4)) * sizeof(double) + 4 * sizeof(unsigned int) + sizeof(int) +
            tasks.size() * sizeof(int2);
  const size_t nsq = 2 * (size_t)L + 4;
  std::vector<double> sqv(2 * nsq, 0.0);
  for (size_t k = 0; k < nsq; ++k) sqv[k] = std::sqrt((double)k);
  for (size_t k = 1; k < nsq; ++k) sqv[nsq + k] = 1.0 / std::sqrt((double)k);
  return cudaMemcpy(w.sqrt_tab, sqv.data(), sqv.size() * sizeof(double), cudaMemcpyHostToDevice);
}

static cudaError_t column_launch(const DeltaWork& w, int L, const float* Uf, const LaneTables* lt, ATiles t,
                                 cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.barrier, 0, 4 * sizeof(unsigned int), st)) != cudaSuccess) return e;
  ColumnParams P;
  P.L = L;
  P.ntasks = w.ntasks;
  P.tasks = w.tasks;
  P.sq = w.sqrt_tab;
  P.rsq = w.sqrt_tab + (2 * (size_t)L + 4);
  P.table = w.table;
  P.counter = w.barrier;
  P.Uf = Uf;
  P.alc = lt ? lt->alc : nullptr;
  P.pc = lt ? lt->pc : nullptr;
  P.A = t.A;
  P.ab2 = lt ? lt->ab2 : nullptr;
  const bool tiles = t.A != nullptr;
  P.extent = tiles ? t.ntiles : (long long)delta_offset(L);
  if (tiles && L > 1024)
    column_tiles_kernel<true><<<lt->col_blocks, kColThreads, kTileSmem, st>>>(P);
  else if (tiles)
    column_tiles_kernel<false><<<lt->col_blocks, kColThreads, kTileSmem, st>>>(P);
  else if (L > 1024)
    column_recursion_kernel<true><<<w.blocks, w.threads, w.smem, st>>>(P);
  else
    column_recursion_kernel<false><<<w.blocks, w.threads, w.smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t column_run(const DeltaWork& w, int L, cudaStream_t st) {
  return column_launch(w, L, nullptr, nullptr, ATiles(), st);
}

void lane_tables_free(LaneTables& t) {
  void* ptrs[] = {t.alc, t.pc, t.alT, t.pT, t.t1m, t.t1e, t.ufT, t.ab2, t.tasks};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  t = LaneTables();
}

cudaError_t lane_tables_setup(LaneTables& t, const DeltaWork& w, int L, int s, const float* Uf, int nC,
                              const long long* abase) {
  cudaError_t e;
  const size_t n = (size_t)L * (L + 1) / 2;
  const int as = s < 0 ? -s : s;
  // tasks (m, kc): column m, degrees of chunk kc from max(m, |s|) on, longest walk first
  std::vector<int2> tasks;
  for (int m = 0; m < L; ++m)
    for (int kc = std::max(m, as) / 32; kc < nC; ++kc) tasks.push_back(make_int2(m, kc));
  auto len = [L](const int2& x) { return std::min(32 * x.y + 31, L - 1) - x.x; };
  std::stable_sort(tasks.begin(), tasks.end(), [&](const int2& x, const int2& y) { return len(x) > len(y); });
  t.ntasks = (int)tasks.size();
  if ((e = dev_malloc(&t.alc, n * sizeof(double))) != cudaSuccess) return e;
  if ((e = dev_malloc(&t.pc, n * sizeof(float))) != cudaSuccess) return e;
  if ((e = dev_malloc(&t.alT, n * sizeof(double))) != cudaSuccess) return e;
  if ((e = dev_malloc(&t.pT, n * sizeof(float))) != cudaSuccess) return e;
  if ((e = dev_malloc(&t.t1m, n * sizeof(double))) != cudaSuccess) return e;
  if ((e = dev_malloc(&t.t1e, n * sizeof(int))) != cudaSuccess) return e;
  if ((e = dev_malloc(&t.ufT, n * sizeof(float))) != cudaSuccess) return e;
  if ((e = dev_malloc(&t.ab2, (size_t)L * sizeof(long long))) != cudaSuccess) return e;
  if ((e = dev_malloc(&t.tasks, std::max<size_t>(tasks.size(), 1) * sizeof(int2))) != cudaSuccess) return e;
  t.bytes = n * (3 * sizeof(double) + sizeof(int) + 3 * sizeof(float)) + (size_t)L * sizeof(long long) +
            tasks.size() * sizeof(int2);
  if (!tasks.empty() &&
      (e = cudaMemcpy(t.tasks, tasks.data(), tasks.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  const double* sq = w.sqrt_tab;
  const double* rsq = w.sqrt_tab + (2 * (size_t)L + 4);
  lane_first_rows_kernel<<<dim3((unsigned)((L + 31) / 32 + 7) / 8, (unsigned)L), 256>>>(L, sq, rsq, t.t1m, t.t1e);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  rescale_tables_kernel<<<(unsigned)((L + 127) / 128), 128>>>(L, sq, rsq, Uf, t.alc, t.pc, t.alT, t.pT, t.ufT);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tile_base_kernel<<<(unsigned)((L + 127) / 128), 128>>>(L, abase, t.ab2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lane_recursion_kernel<false>, kColThreads, 0)) !=
        cudaSuccess)
      return e;
    t.blocks = sms * std::max(1, std::min(per_sm, SSHT_LANE_CTAS));
    const void* fns[2] = {(const void*)column_tiles_kernel<false>, (const void*)column_tiles_kernel<true>};
    for (const void* fn : fns) {
      if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
        return e;
    }
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[L > 1024 ? 1 : 0], kColThreads, kTileSmem)) !=
        cudaSuccess)
      return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    t.col_blocks = sms * std::min(per_sm, SSHT_COLUMN_CTAS);
  }
  if ((e = cudaFuncSetAttribute(lane_recursion_kernel<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(lane_recursion_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
    return e;
  return cudaDeviceSynchronize();
}

cudaError_t column_run_inverse_tiles(const DeltaWork& w, const LaneTables& t, int L, int s, InvTiles it,
                                     cudaStream_t st) {
  if (!it.A || !it.ibase || !t.alT || w.method != kDeltaColumn) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.barrier, 0, 4 * sizeof(unsigned int), st)) != cudaSuccess) return e;
  LaneParams P;
  P.L = L;
  P.as = s < 0 ? -s : s;
  P.nI = it.nI;
  P.ntasks = t.ntasks;
  P.tasks = t.tasks;
  P.alpha = t.alT;
  P.p = t.pT;
  P.t1m = t.t1m;
  P.t1e = t.t1e;
  P.ufT = t.ufT;
  P.A = it.A;
  P.ibase = it.ibase;
  P.counter = w.barrier;
  P.ntiles = it.ntiles;
  if (L > 1024)
    lane_recursion_kernel<true><<<t.blocks, kColThreads, 0, st>>>(P);
  else
    lane_recursion_kernel<false><<<t.blocks, kColThreads, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t column_run_tiles(const DeltaWork& w, const LaneTables& lt, int L, const float* Uf, ATiles t,
                             cudaStream_t st) {
  if (!t.A || !lt.ab2 || !lt.alc || !Uf || w.method != kDeltaColumn) return cudaErrorInvalidValue;
  return column_launch(w, L, Uf, &lt, t, st);
}

SSHT_BOUNDS_TU(delta_column)

}  // namespace ssht
