// Delta^l = d^l(pi/2) for l = 0 .. L-1 by the Risbo recursion (the recursion the paper
// uses, Sec. 2.2), FP64, on the symmetry-reduced octant 0 <= n <= m <= l.
//
// One half step couples d^{j-1/2} with the spin-1/2 matrix [[p,-q],[q,p]], p = q = 1/sqrt2:
//   d^j_{mn} = p/(2j) [ sqrt(j+m) ( sqrt(j+n) X(m-1/2, n-1/2) - sqrt(j-n) X(m-1/2, n+1/2) )
//                     + sqrt(j-m) ( sqrt(j+n) X(m+1/2, n-1/2) + sqrt(j-n) X(m+1/2, n+1/2) ) ]
// with X = d^{j-1/2} (zero outside |index| <= j - 1/2).  Entries outside the stored octant
// are read through the symmetry relations
//   d_{mn} = (-1)^{m-n} d_{nm}            (transpose; from eqn wignerd_sym3, any j),
//   d_{mn} = (-1)^{m-n} d_{-m,-n}         (eqn wignerd_sym1),
//   Delta^l_{m,-n} = (-1)^{l+m} Delta^l_{mn}  (eqn wignerd_sym1 with eqn wignerd_sym2, integer l).
//
// Storage.  The octant slab of integer degree l keeps row m (0 <= m <= l) with the columns
// n = -1 .. m+1, the two extra ones holding Delta_{m,-1} and Delta_{m,m+1} (given by the symmetry
// relations), so that every stencil read is a plain indexed load; the half-integer rows are laid
// out the same way in shared memory.
//
// Parallel layout.  One cooperative persistent grid walks l.  For the step l -> l+1 the rows
// of the new integer slab are split over the CTAs by a partition made on the host that minimises
// the largest share of 32-column segments (a warp computes one segment per instruction stream),
// or, without a host table, by equal shares made in the kernel.  A CTA that owns integer rows
// [r0, r1) works through them in chunks [c0, c1) sized to its shared memory: it copies the padded
// rows [c0-1, c1] of degree l from global memory into shared memory, computes the half-integer
// rows [c0-1, c1-1], then the integer rows [c0, c1), which go to the next slab (global) and to
// shared memory.  Warp 0 then publishes "degree l+1 done" in the CTA's flag word and waits for the
// flags of the next step while the other warps write the rows to the quadrant table from shared
// memory, both orientations coalesced.  A CTA waits only for the CTAs that produced the rows of
// degree l it reads (which are also all the readers of the slab rows it overwrites): no grid-wide
// barrier per degree.  Every wait spins at most one second, then latches a status bit, raises the
// abort flag and leaves the kernel; the other CTAs leave at their next wait.
#include "ssht_internal.h"

#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>
#include <vector>

namespace ssht {
namespace {

#ifndef SSHT_RISBO_THREADS
#define SSHT_RISBO_THREADS 512
#endif
#ifndef SSHT_RISBO_MARK
#define SSHT_RISBO_MARK(k)  // phase boundary: 1 waited, 2 staged, 3 half step, 4 integer step, 5 table written
#endif
constexpr int kThreads = SSHT_RISBO_THREADS;
static_assert(kThreads >= 64 && kThreads % 32 == 0, "warp 0 polls and publishes while the other warps write the table");

struct RisboParams {
  int L;
  double* table;
  double* slab0;
  double* slab1;
  const double* sq;         // sqrt(k)
  const double* rsq;        // 1/sqrt(k), k >= 1
  unsigned int* counter;    // [0] barrier counter, [1] abort flag, [4 + c] degree done by CTA c (reset before launch)
  const int4* part;         // per step l and CTA: r0, r1, o0, o1 (host-made), or null: computed here
  int* status;              // latched status bits
  long long limit_ns;       // spin limit of every wait
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier with a one-second spin limit.  Returns false if this CTA must stop.  While
// thread 0 waits, thread 32 (another warp) runs `side()`.
template <typename Side>
__device__ bool grid_barrier(unsigned int* counter, unsigned int target, int* status, long long limit_ns, Side side) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
    int good = 1;
    const unsigned long long t0 = globaltimer_ns();
    unsigned int spins = 0;
    while (ld_acquire_u32(counter) < target) {
      if ((++spins & 63u) == 0u) {
        if (*(volatile unsigned int*)(counter + 1) != 0u) { good = 0; break; }
        if ((long long)(globaltimer_ns() - t0) > limit_ns) {
          atomicOr(status, kStatusBarrierTimeout);
          atomicExch(counter + 1, 1u);
          good = 0;
          break;
        }
      }
    }
    __threadfence();
    ok = good;
  } else if (threadIdx.x == 32) {
    side();
  }
  __syncthreads();
  return ok != 0;
}

__host__ __device__ __forceinline__ long long tri_ll(long long m) { return m * (m + 1) / 2; }

// Padded row layout shared by the octant slabs (global) and the staged rows (shared memory):
// row m holds columns n = -1 .. m+1 at po(m) + n + 1, po(m) = m(m+5)/2 (row m has m+3 slots).
// The two extra columns carry Delta_{m,-1} and Delta_{m,m+1}, which the symmetry relations give
// from stored entries; with them every stencil read of a step is a plain indexed load.
__host__ __device__ __forceinline__ long long po(long long m) { return m * (m + 5) / 2; }

// Segments of 32 columns in rows 1 .. n of lengths 1 .. n: sum_{k=1}^{n} ceil(k/32).
__host__ __device__ __forceinline__ long long segF(long long n) {
  const long long q = n >> 5, r = n & 31;
  return 16 * q * (q + 1) + r * (q + 1);
}

// Work of integer rows [0, m) of a step, half rows included, in 32-column segments: row k has
// k + 3 half-integer and k + 2 integer columns (each step's update reads one column more than
// it writes).
__host__ __device__ __forceinline__ long long row_cost(long long m) { return segF(m + 2) - 2 + segF(m + 1) - 1; }

// Row m0 of the split of rows [0, rows) with cut o of nb: the smallest m with
// row_cost(m) >= floor(row_cost(rows) * o / nb).
__host__ __device__ __forceinline__ int cut_row(int rows, int o, int nb) {
  const long long x = row_cost(rows) * o / nb;
  int a = 0, b = rows;
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (row_cost(mid) >= x) b = mid; else a = mid + 1;
  }
  return a;
}

// Rows [r0, r1) of the integer slab of degree lp (rows 0 .. lp) owned by CTA cta of nb.
__host__ __device__ __forceinline__ void cta_rows(int lp, int cta, int nb, int* r0, int* r1) {
  *r0 = cut_row(lp + 1, cta, nb);
  *r1 = cut_row(lp + 1, cta + 1, nb);
}

// The CTA that owns row `row` of degree l: the largest o with cut_row(l + 1, o, nb) <= row.
__host__ __device__ __forceinline__ int row_owner(int l, int row, int nb) {
  const long long S = row_cost(l + 1);
  const long long o = ((row_cost(row) + 1) * nb + S - 1) / S - 1;
  return (int)(o < nb - 1 ? o : nb - 1);
}

// v with its sign flipped when neg is set, by integer ops on the sign bit (a multiplication by
// -1 would cost an FP64 instruction).
__device__ __forceinline__ double flip(double v, bool neg) {
  return __hiloint2double(__double2hiint(v) ^ (neg ? (int)0x80000000 : 0), __double2loint(v));
}

// Shared-memory bytes of the copies of the sqrt and reciprocal sqrt tables (2L + 4 entries each)
// that follow a CTA's chunk area, rounded to 16.
__host__ __device__ constexpr size_t sq_smem_bytes(long long L) { return (2 * (2 * L + 4) * 8 + 15) / 16 * 16; }

// Doubles of one padded octant slab for band-limit L (rows 0 .. L, with slack).
__host__ __device__ constexpr size_t slab_doubles(long long L) { return (size_t)((L + 2) * (L + 7) / 2 + 2); }

// Shared-memory doubles for integer rows [c0, c1) of degree l+1 made from degree l: integer rows
// [Alo, Ahi + 1] and half rows [Alo - 1, c1 - 1] (row Alo - 1 has two slots), all padded, the new
// rows [c0, c1) packed (for the table writes), and the row factors of both steps.
__host__ __device__ __forceinline__ long long chunk_need(int l, int c0, int c1) {
  const int Alo = c0 > 0 ? c0 - 1 : 0;
  const int Ahi = (c1 - 1 < l) ? c1 - 1 : l;
  return (po(Ahi + 2) - po(Alo)) + 2 + (po(c1) - po(Alo)) + (tri_ll(c1) - tri_ll(c0)) + 2 * (Ahi - Alo + 1) +
         2 * (c1 - c0);
}

// 32-bit forms of the index maps for the kernel (all values stay below 2^31 for L <= 2048).
__device__ __forceinline__ int po32(int m) { return m * (m + 5) / 2; }
__device__ __forceinline__ int tri32(int m) { return m * (m + 1) / 2; }
__device__ __forceinline__ int segF32(int n) {
  const int q = n >> 5, r = n & 31;
  return 16 * q * (q + 1) + r * (q + 1);
}
// Largest n >= 0 with segF(n) <= t (t >= 0): the 32-column block q from a square root, then the
// column in it by one division.
__device__ __forceinline__ int segF_inv(int t) {
  int q = (int)((sqrtf(1.0f + 0.25f * (float)t) - 1.0f) * 0.5f);
  if (q < 0) q = 0;
  while (q > 0 && 16 * q * (q + 1) > t) --q;
  while (16 * (q + 1) * (q + 2) <= t) ++q;
  int r = (t - 16 * q * (q + 1)) / (q + 1);
  return 32 * q + (r < 31 ? r : 31);
}

// A warp's share of the 32-column segments of rows [lo, hi] whose row x has x + add columns:
// the first row x, the segment in it, and the number of segments; the shares of the warps of a
// CTA are contiguous and equal to within one.
struct SegRange {
  int x, seg, count;
};
__device__ __forceinline__ SegRange warp_segments(int lo, int hi, int add, int warp, int nwarps) {
  const int base = segF32(lo + add - 1);
  const int S = segF32(hi + add) - base;
  const int s0 = S * warp / nwarps, s1 = S * (warp + 1) / nwarps;
  int x = segF_inv(base + s0) - add + 1;
  if (x > hi) x = hi;
  if (x < lo) x = lo;
  SegRange r;
  r.x = x;
  r.seg = s0 - (segF32(x + add - 1) - base);
  r.count = s1 - s0;
  return r;
}

// Step l -> l + 1 of CTA cta: owned rows q[0], q[1] of degree l + 1, and the CTAs q[2] .. q[3]
// that produced the degree-l rows [r0 - 2, r1 + 1]: the rows staged here, and the rows whose
// producers also read (one step earlier) the slab rows this CTA overwrites, pad slots included.
__host__ __device__ inline void step_partition(int l, int cta, int nb, int* q) {
  int r0, r1;
  cta_rows(l + 1, cta, nb, &r0, &r1);
  q[0] = r0;
  q[1] = r1;
  const int a = r0 - 2 > 0 ? r0 - 2 : 0, b = r1 + 1 < l ? r1 + 1 : l;
  q[2] = row_owner(l, a, nb);
  q[3] = row_owner(l, b, nb);
}

// Warp 0 waits until every flag of CTAs [o0, o1] has reached `degree` (acquire), one lane per
// flag so that the polls overlap, one second at most; returns (to every lane) whether to go on.
__device__ bool poll_flags(const unsigned int* done, int o0, int o1, unsigned int degree, unsigned int* abort_flag,
                           int* status, long long limit_ns) {
  const int lane = threadIdx.x & 31;
  int good = 1;
  const unsigned long long t0 = globaltimer_ns();
  for (int base = o0; base <= o1 && good; base += 32) {
    const int o = base + lane;
    unsigned int spins = 0;
    while (true) {
      const bool mine = o > o1 || ld_acquire_u32(done + o) >= degree;
      if (__all_sync(0xffffffffu, mine)) break;
      if ((++spins & 63u) == 0u) {
        int stop = 0;
        if (lane == 0) {
          if (*(volatile unsigned int*)abort_flag != 0u) {
            stop = 1;
          } else if ((long long)(globaltimer_ns() - t0) > limit_ns) {
            atomicOr(status, kStatusBarrierTimeout);
            atomicExch(abort_flag, 1u);
            stop = 1;
          }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) {
          good = 0;
          break;
        }
      }
    }
  }
  return good != 0;
}

// poll_flags by warp 0, then a barrier; all threads learn whether to go on.
__device__ bool wait_flags(const unsigned int* done, int o0, int o1, unsigned int degree, unsigned int* abort_flag,
                           int* status, long long limit_ns) {
  __shared__ int ok;
  if (threadIdx.x < 32) {
    const bool good = poll_flags(done, o0, o1, degree, abort_flag, status, limit_ns);
    if (threadIdx.x == 0) ok = good ? 1 : 0;
  }
  __syncthreads();
  return ok != 0;
}

// At most 72 registers a thread (one CTA of 512 threads per SM): the rest of the register file
// stays free for the kernels that share the SMs from other streams.
__global__ void __maxnreg__(72) risbo_kernel(RisboParams P, long long cap) {
  extern __shared__ double smem[];
  // Per step l -> l + 1 (slot l & 1): owned rows r0, r1 of degree l + 1, the CTAs o0..o1 that
  // produced the degree-l rows read here, and the step scales p/(2j).
  __shared__ int s_par[2][4];
  __shared__ double s_sc[2][2];
  // The step whose flags warp 0 already waited for at the end of the previous step (-1: none,
  // -2: that wait gave up).
  __shared__ int s_pre;
  const int nb = gridDim.x;
  const int cta = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // sqrt(k) and 1/sqrt(k) from shared memory (the column and row factors): copied after the
  // chunk area, published by the grid barrier's first __syncthreads.
  double* sq_s = smem + cap;
  for (int k = threadIdx.x; k < 2 * P.L + 4; k += blockDim.x) {
    sq_s[k] = P.sq[k];
    sq_s[2 * P.L + 4 + k] = P.rsq[k];
  }
  const double* __restrict__ sq = sq_s;
  const double* __restrict__ rsq = sq_s + 2 * P.L + 4;
  // Thread 32 makes the next step's parameters while the step runs; the partition entry comes
  // from a register loaded a step earlier, so that no global load or FP64 division sits in a
  // step (1/(2j) = (1/sqrt(2j))^2 from the shared table).
  int4 part_next = make_int4(0, 0, 0, 0);
  auto load_part = [&](int l) { return P.part ? __ldg(&P.part[(size_t)l * nb + cta]) : make_int4(0, 0, 0, 0); };
  auto params = [&](int l, int4 v) {
    int* q = s_par[l & 1];
    const int lp = l + 1;
    if (P.part) {
      q[0] = v.x;
      q[1] = v.y;
      q[2] = v.z;
      q[3] = v.w;
    } else {
      step_partition(l, cta, nb, q);
    }
    const double r1 = rsq[2 * l + 1], r2 = rsq[2 * lp];
    s_sc[l & 1][0] = 0.70710678118654752440 * (r1 * r1);
    s_sc[l & 1][1] = 0.70710678118654752440 * (r2 * r2);
  };

  if (threadIdx.x == 0) s_pre = -1;
  unsigned int* done = P.counter + 4;
  if (cta == 0 && threadIdx.x < 3) {  // degree 0: row 0 = (Delta_{0,-1}, Delta_00, Delta_01) = (0, 1, 0)
    P.slab0[threadIdx.x] = threadIdx.x == 1 ? 1.0 : 0.0;
    if (threadIdx.x == 0) P.table[0] = 1.0;
  }
  if (!grid_barrier(P.counter, nb, P.status, P.limit_ns, [&] {
        params(0, load_part(0));
        if (P.L > 2) part_next = load_part(1);
      }))
    return;
  for (int l = 0; l + 1 < P.L; ++l) {
    __syncthreads();  // params(l) visible; every thread is done with step l - 1
    if (s_pre == -2) return;
    const int lp = l + 1;
    const int r0 = s_par[l & 1][0], r1 = s_par[l & 1][1];
    const int o0 = s_par[l & 1][2], o1 = s_par[l & 1][3];
    const double sc = s_sc[l & 1][0], sc2 = s_sc[l & 1][1];
    if (threadIdx.x == 32 && l + 2 < P.L) {
      params(l + 1, part_next);
      if (l + 3 < P.L) part_next = load_part(l + 2);
    }
    if (r0 >= r1) {  // nothing owned at this degree: nothing to wait for or to publish but progress
      if (threadIdx.x == 0) atomicExch(done + cta, (unsigned)lp);
      continue;
    }
    if (s_pre != l && !wait_flags(done, o0, o1, (unsigned)l, P.counter + 1, P.status, P.limit_ns)) return;
    SSHT_RISBO_MARK(1);
    const double* __restrict__ Yg = (l & 1) ? P.slab1 : P.slab0;
    double* __restrict__ Yn = (l & 1) ? P.slab0 : P.slab1;
    double* __restrict__ T = P.table + (size_t)((long long)lp * (lp + 1) * (2 * lp + 1) / 6);
    for (int c0 = r0; c0 < r1;) {
      // The whole share in one chunk when it fits (the usual case), else the largest c1 that fits.
      int c1 = r1;
      if (chunk_need(l, c0, r1) > cap) {
        int lo = c0 + 1, hi = r1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (chunk_need(l, c0, mid) <= cap) lo = mid; else hi = mid - 1;
        }
        c1 = lo;
      }
      const int Alo = c0 > 0 ? c0 - 1 : 0;
      const int Ahi = (c1 - 1 < l) ? c1 - 1 : l;   // half rows computed here
      const int Ytop = (Ahi + 1 < l) ? Ahi + 1 : l; // integer rows staged from degree l
      const int ybase = po32(Alo);
      const int ycount = po32(Ytop + 1) - ybase;
      const int z0 = tri32(c0);
      double* __restrict__ Ys = smem;                              // integer rows [Alo, Ahi + 1]
      double* __restrict__ Xs = smem + (po32(Ahi + 2) - ybase);    // half rows [Alo - 1, c1 - 1]
      double* __restrict__ Zs = Xs + 2 + (po32(c1) - ybase);       // new rows [c0, c1), packed
      double* __restrict__ Rh = Zs + (tri32(c1) - z0);             // half-step row factors, 2 per row
      double* __restrict__ Ri = Rh + 2 * (Ahi - Alo + 1);          // integer-step row factors
      if (c0 > r0) __syncthreads();  // the previous chunk is done with shared memory
      // Stage the contiguous padded rows [Alo, Ytop] of degree l (asynchronous copies, all in
      // flight together).  Rows beyond l are zero: the integer row l + 1 (when Ahi = l) and the
      // half row l + 1 (when c1 - 1 = l + 1), whose padded neighbour slot in row l is zero too.
      for (int i = threadIdx.x; i < ycount; i += blockDim.x) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(Ys + i);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(Yg + ybase + i) : "memory");
      }
      if (Ytop < Ahi + 1)
        for (int i = threadIdx.x; i < l + 4; i += blockDim.x) Ys[po32(l + 1) - ybase + i] = 0.0;
      if (c1 - 1 > l)
        for (int i = threadIdx.x; i < l + 4; i += blockDim.x) Xs[2 + po32(l + 1) - ybase + i] = 0.0;
      // Row factors.  The step factors of half row A are ra = sqrt(j+a) p/(2j) and
      // rb = sqrt(j-a) p/(2j) (j+a = l+A+1, j-a = l-A), of integer row m ia = sqrt(j+m) p/(2j)
      // and ib = sqrt(j-m) p/(2j) (j = lp).  Half row A is kept divided by ra(A) (row -1 by
      // ra(0)), so a half-step update needs kappa = rb/ra only; the integer step multiplies by
      // alpha = ia(m) ra(m-1) and combines the half rows with kappa = ib ra(m) / (ia ra(m-1)).
      for (int A = Alo + (int)threadIdx.x; A <= Ahi; A += blockDim.x) {
        Rh[2 * (A - Alo)] = sq[l - A] * rsq[l + A + 1];                     // rb / ra
        Rh[2 * (A - Alo) + 1] = A > 0 ? sq[l + A + 1] * rsq[l + A] : 1.0;  // ra(A) / ra(A-1)
      }
      for (int m = c0 + (int)threadIdx.x; m < c1; m += blockDim.x) {
        Ri[2 * (m - c0)] = sq[lp + m] * sc2 * ((m > 0 ? sq[l + m] : sq[l + 1]) * sc);
        Ri[2 * (m - c0) + 1] = m > 0 ? (sq[lp - m] * sq[l + m + 1]) * (rsq[lp + m] * rsq[l + m]) : 1.0;
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      SSHT_RISBO_MARK(2);
      // Half step l -> l + 1/2 (2j = 2l + 1), half rows A in [Alo, Ahi], columns B in [0, A+1]
      // (a = A + 1/2, b = B - 1/2): j+a = l+A+1, j-a = l-A, j+b = l+B, j-b = l+1-B.  With
      // P(c) = Y(A, c) + kappa Y(A+1, c) and Q(c) = kappa Y(A+1, c) - Y(A, c),
      //   X(A, B) / ra(A) = sqrt(j+b) P(B-1) + sqrt(j-b) Q(B):
      // lane i forms P and Q of column i - 1 and takes P of the column before from its left
      // neighbour (lane 0 from lane 31 of the warp's previous segment).
      {
        const SegRange w = warp_segments(Alo, Ahi, 3, warp, nwarps);
        int A = w.x, seg = w.seg;
        int yo = po32(A) - ybase;  // row A of Ys from column -1; half row A of Xs is at 2 + yo
        double kap = Rh[2 * (A - Alo)], rat = Rh[2 * (A - Alo) + 1];
        double carry = 0.0;
        if (w.count > 0 && seg > 0) {
          const int i = seg * 32 - 1;
          carry = fma(kap, Ys[yo + A + 3 + i], Ys[yo + i]);
        }
        for (int k = 0; k < w.count; ++k) {
          const int i = seg * 32 + lane;  // column i - 1
          double P = 0.0, Q = 0.0;
          if (i <= A + 2) {
            const double y0 = Ys[yo + i], y1 = Ys[yo + A + 3 + i];
            P = fma(kap, y1, y0);
            Q = fma(kap, y1, -y0);
          }
          double Pm = __shfl_up_sync(0xffffffffu, P, 1);
          const double P31 = __shfl_sync(0xffffffffu, P, 31);
          if (lane == 0) Pm = carry;
          carry = P31;
          if (i >= 1 && i <= A + 2) {
            const int B = i - 1;
            const double v = fma(sq[l + 1 - B], Q, sq[l + B] * Pm);
            double* xr = Xs + 2 + yo;
            xr[B] = v;
            if (B == A) {
              if (A > Alo) xr[-1] = -v * rat;            // pad of row A-1, in its scale: X(A-1, A+1) = -X(A, A)
              else if (A == 0) Xs[1] = flip(v, true);    // X(-1/2, 1/2) = -X(1/2, -1/2)
            }
            if (A == 0 && B == 1) Xs[0] = v;             // X(-1/2, -1/2) = X(1/2, 1/2)
          }
          if (++seg * 32 > A + 2) {
            yo += A + 3;
            ++A;
            seg = 0;
            if (A <= Ahi) {
              kap = Rh[2 * (A - Alo)];
              rat = Rh[2 * (A - Alo) + 1];
            }
          }
        }
      }
      if (c1 - 1 > l && threadIdx.x == 0) Xs[2 + (po32(l) - ybase) + l + 2] = 0.0;  // X(l, l+2) = -X(l+1, l+1) = 0
      __syncthreads();
      SSHT_RISBO_MARK(3);
      // Integer step l + 1/2 -> lp (2j = 2 lp), rows m in [c0, c1), columns n in [0, m]:
      // j+m = lp+m, j-m = lp-m, j+n = lp+n, j-n = lp-n; X(m - 1/2, .) is half row m - 1.  With
      // P(c) = X'(m-1, c) + kappa X'(m, c) and Q(c) = kappa X'(m, c) - X'(m-1, c) (X' the stored,
      // divided half rows), Delta_{mn} = alpha (sqrt(j+n) P(n) + sqrt(j-n) Q(n+1)): lane i forms P
      // and Q of column i and writes column n = i - 1.
      {
        const SegRange w = warp_segments(c0, c1 - 1, 2, warp, nwarps);
        int m = w.x, seg = w.seg;
        int xo = 2 + po32(m) - ybase;  // half row m in Xs (row m - 1 starts m + 2 earlier; row -1 at 0)
        int zo = tri32(m) - z0;
        double* yr = Yn + po32(m);
        double al = Ri[2 * (m - c0)], kap = Ri[2 * (m - c0) + 1];
        double carry = 0.0;
        if (w.count > 0 && seg > 0) {
          const int i = seg * 32 - 1;
          carry = fma(kap, Xs[xo + i], Xs[(m > 0 ? xo - (m + 2) : 0) + i]);
        }
        for (int k = 0; k < w.count; ++k) {
          const int i = seg * 32 + lane;
          double P = 0.0, Q = 0.0;
          if (i <= m + 1) {
            const double x0 = Xs[(m > 0 ? xo - (m + 2) : 0) + i], x1 = Xs[xo + i];
            P = fma(kap, x1, x0);
            Q = fma(kap, x1, -x0);
          }
          double Pm = __shfl_up_sync(0xffffffffu, P, 1);
          const double P31 = __shfl_sync(0xffffffffu, P, 31);
          if (lane == 0) Pm = carry;
          carry = P31;
          if (i >= 1 && i <= m + 1) {
            const int n = i - 1;
            const double v = al * fma(sq[lp - n], Q, sq[lp + n] * Pm);
            yr[n + 1] = v;
            if (n == 1) yr[0] = flip(v, ((lp + m) & 1) != 0);            // Delta_{m,-1} = (-1)^{l+m} Delta_{m,1}
            if (n + 1 == m) {
              yr[-1] = flip(v, true);                                     // Delta_{m-1,m} = -Delta_{m,m-1}
              if (m == 1) yr[-3] = flip(v, (lp & 1) == 0);                // Delta_{0,-1} = (-1)^{l+1} Delta_{1,0}
            }
            if (n == m && m == lp) yr[m + 2] = 0.0;                       // Delta_{l,l+1} = 0
            Zs[zo + n] = v;
          }
          if (++seg * 32 > m + 1) {
            xo += m + 3;
            zo += m + 1;
            yr += m + 3;
            ++m;
            seg = 0;
            if (m < c1) {
              al = Ri[2 * (m - c0)];
              kap = Ri[2 * (m - c0) + 1];
            }
          }
        }
      }
      __syncthreads();
      SSHT_RISBO_MARK(4);
      if (warp == 0) {
        if (c1 == r1) {
          // The slab rows of this CTA are complete: publish them, then wait for the flags of the
          // next step while the other warps write the table.
          if (lane == 0) {
            __threadfence();
            atomicExch(done + cta, (unsigned)lp);
          }
          __syncwarp();
          if (l + 2 < P.L) {
            const int* q = s_par[(l + 1) & 1];  // made by thread 32 before this step's barriers
            if (q[0] < q[1]) {
              const bool good = poll_flags(done, q[2], q[3], (unsigned)lp, P.counter + 1, P.status, P.limit_ns);
              if (lane == 0) s_pre = good ? lp : -2;
            }
          }
        }
      } else {
        // Quadrant table from shared memory (warps 1 ..): rows T[m][n] = Delta_{mn} (n <= m) ...
        {
          const SegRange w = warp_segments(c0, c1 - 1, 1, warp - 1, nwarps - 1);
          int m = w.x, seg = w.seg;
          int zo = tri32(m) - z0;
          double* trow = T + (size_t)m * (lp + 1);
          for (int k = 0; k < w.count; ++k) {
            const int n = seg * 32 + lane;
            if (n <= m) trow[n] = Zs[zo + n];
            if (++seg * 32 > m) {
              zo += m + 1;
              trow += lp + 1;
              ++m;
              seg = 0;
            }
          }
        }
        // ... and T[n][m] = (-1)^{m-n} Delta_{mn} (n < m): for each table row n, the columns
        // m in [max(c0, n+1), c1) are contiguous.
        {
          const int width = c1 - c0;
          const int items = (c1 - 1) * width;  // n in [0, c1 - 1)
          const float inv_w = 1.0f / (float)width;
          for (int i = (int)threadIdx.x - 32; i < items; i += (int)blockDim.x - 32) {
            int n = (int)(((float)i + 0.5f) * inv_w);
            int j = i - n * width;
            if (j < 0) { --n; j += width; } else if (j >= width) { ++n; j -= width; }
            const int m = c0 + j;
            if (m > n) T[(size_t)n * (lp + 1) + m] = flip(Zs[tri32(m) - z0 + n], ((m - n) & 1) != 0);
          }
        }
      }
      SSHT_RISBO_MARK(5);
      c0 = c1;
    }
  }
}

// U[tri(l) + m'] = sqrt((2l+1)/4pi) Delta^l_{m',-s} for l >= |s|, 0 otherwise.
__global__ void spin_column_kernel(const double* __restrict__ table, int L, int s, double* __restrict__ U,
                                   float* __restrict__ Uf) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= tri_ll(L)) return;
  int l = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
  while (l > 0 && tri_ll(l) > e) --l;
  while (tri_ll(l + 1) <= e) ++l;
  const int mp = (int)(e - tri_ll(l));
  const int as = s < 0 ? -s : s;
  double v = 0.0;
  if (l >= as) {
    const double* T = table + (size_t)((long long)l * (l + 1) * (2 * l + 1) / 6);
    const double d = T[(size_t)mp * (l + 1) + as];
    // Delta_{m',-s}: for s <= 0 the column -s >= 0 is stored; for s > 0 use eqn wignerd_sym6.
    v = (s > 0 && ((l + mp) & 1)) ? -d : d;
    v *= sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846));
  }
  U[e] = v;
  Uf[e] = (float)v;
}

}  // namespace

// Host partition of the integer rows 0 .. l+1 of step l -> l + 1 over nb CTAs into contiguous
// ranges cuts[c] .. cuts[c+1] that minimise the largest share.  A share costs the 32-column
// segments of its integer rows and their half rows, one more per row, plus the half row just
// below its first row, which it computes too (the neighbour computes it as well).  Binary search on the largest share
// with first-fit packing; CTAs left over get empty ranges at the top.
static void optimal_cuts(int l, int nb, int* cuts) {
  const int rows = l + 2;
  auto seg = [](long long n) { return (n + 31) / 32; };
  std::vector<long long> pre(rows + 1, 0);
  // (+1 per row: the fixed cost of starting a row, which counts for the many short rows)
  for (int m = 0; m < rows; ++m) pre[m + 1] = pre[m] + (m <= l ? seg(m + 3) : 0) + seg(m + 2) + 1;
  auto share = [&](int a, int b) { return pre[b] - pre[a] + (a > 0 ? seg(a + 2) : 0); };
  auto pack = [&](long long T, int* out) {
    int a = 0, c = 0;
    while (a < rows) {
      if (c == nb) return false;
      int b = a + 1;
      if (share(a, b) > T) return false;
      while (b < rows && share(a, b + 1) <= T) ++b;
      if (out) out[c] = a;
      a = b;
      ++c;
    }
    if (out) {
      for (int k = c; k <= nb; ++k) out[k] = rows;
    }
    return true;
  };
  long long lo = 1, hi = share(0, rows);
  while (lo < hi) {
    const long long mid = (lo + hi) / 2;
    if (pack(mid, nullptr)) hi = mid; else lo = mid + 1;
  }
  pack(lo, cuts);
}

static cudaError_t risbo_setup(DeltaWork& w, int L, int device) {
  cudaError_t e;
  int sms = 0, per_sm = 0, smem_optin = 0;
  w.method = kDeltaRisbo;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess) return e;
  w.threads = kThreads;
  w.blocks = sms;  // one CTA per SM
  // Shared memory: what the largest single-chunk share of any degree needs (so no degree is
  // split into chunks), at most 200 KB.  Staying small leaves room on each SM for the kernels
  // that run beside the recursion on other streams.
  const int nb = w.blocks, steps = L > 1 ? L - 1 : 0;
  std::vector<int> cuts((size_t)(steps > 0 ? steps : 1) * (nb + 1));
  for (int l = 0; l < steps; ++l) optimal_cuts(l, nb, &cuts[(size_t)l * (nb + 1)]);
  {
    long long need = 0;
    for (int l = 0; l < steps; ++l)
      for (int c = 0; c < nb; ++c) {
        const int r0 = cuts[(size_t)l * (nb + 1) + c], r1 = cuts[(size_t)l * (nb + 1) + c + 1];
        if (r0 < r1) need = std::max(need, chunk_need(l, r0, r1));
      }
    const size_t want = (((size_t)need + 16) * sizeof(double) + 1023) / 1024 * 1024;
    const size_t limit = (size_t)std::min(smem_optin - 1024, 200 * 1024) - sq_smem_bytes(L);
    const size_t chunk = std::min(want, limit);
    w.cap = (long long)(chunk / sizeof(double));
    w.smem = chunk + sq_smem_bytes(L);  // the chunk area, then the sqrt table
  }
  // Every chunk holds at least one row: the widest single-row chunk (last degree) must fit.
  for (int m = 0; m < L; ++m)
    if (chunk_need(L - 2 > 0 ? L - 2 : 0, m, m + 1) > w.cap) return cudaErrorInvalidValue;
  // The attribute is process-wide and an upper bound: always the cap, so that plans of other
  // sizes (and the no-allocation entry point) can launch with their own amounts.
  if ((e = cudaFuncSetAttribute(risbo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                std::min(smem_optin - 1024, 200 * 1024))) != cudaSuccess)
    return e;
  if ((e = prefer_shared(risbo_kernel)) != cudaSuccess || (e = prefer_shared(spin_column_kernel)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, risbo_kernel, kThreads, w.smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  if ((e = dev_malloc(&w.table, delta_offset(L) * sizeof(double))) != cudaSuccess) return e;
  if ((e = dev_malloc(&w.slab[0], slab_doubles(L) * sizeof(double))) != cudaSuccess) return e;
  if ((e = dev_malloc(&w.slab[1], slab_doubles(L) * sizeof(double))) != cudaSuccess) return e;
  if ((e = dev_malloc(&w.sqrt_tab, 2 * (2 * (size_t)L + 4) * sizeof(double))) != cudaSuccess) return e;
  if ((e = dev_malloc(&w.barrier, (4 + (size_t)w.blocks) * sizeof(unsigned int))) != cudaSuccess) return e;
  if ((e = dev_malloc(&w.status, sizeof(int))) != cudaSuccess) return e;
  {
    // the partition of every step, made once here (the kernel reads one int4 per step)
    const size_t n = (size_t)(steps > 0 ? steps : 1) * nb;
    std::vector<int4> part(n, make_int4(0, 0, 0, 0));
    // the CTA whose range of step l - 1 (which made degree l) holds `row`
    auto owner = [&](int l, int row) {
      if (l == 0) return 0;  // degree 0 comes from the initial barrier
      const int* cp = &cuts[(size_t)(l - 1) * (nb + 1)];
      int c = (int)(std::upper_bound(cp, cp + nb + 1, row) - cp) - 1;
      return c < 0 ? 0 : (c > nb - 1 ? nb - 1 : c);
    };
    for (int l = 0; l < steps; ++l)
      for (int c = 0; c < nb; ++c) {
        const int r0 = cuts[(size_t)l * (nb + 1) + c], r1 = cuts[(size_t)l * (nb + 1) + c + 1];
        // degree-l rows [r0 - 2, r1 + 1]: the rows staged here, and the rows whose producers also
        // read (one step earlier) the slab rows this CTA overwrites, pad slots included
        const int a = r0 - 2 > 0 ? r0 - 2 : 0, b = r1 + 1 < l ? r1 + 1 : l;
        part[(size_t)l * nb + c] = r0 < r1 ? make_int4(r0, r1, owner(l, a), owner(l, b)) : make_int4(r0, r0, 0, -1);
      }
    if ((e = dev_malloc(&w.part, n * sizeof(int4))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(w.part, part.data(), n * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    w.bytes_part = n * sizeof(int4);
  }
  if ((e = cudaMemset(w.status, 0, sizeof(int))) != cudaSuccess) return e;
  w.bytes = (delta_offset(L) + 2 * slab_doubles(L) + 2 * (2 * (size_t)L + 4)) * sizeof(double) +
            (4 + (size_t)w.blocks) * sizeof(unsigned int) + sizeof(int) + w.bytes_part;
  // sqrt(k), then 1/sqrt(k) (entry 0 unused), k < 2L + 4
  const size_t nsq = 2 * (size_t)L + 4;
  std::vector<double> sq(2 * nsq, 0.0);
  for (size_t k = 0; k < nsq; ++k) sq[k] = std::sqrt((double)k);
  for (size_t k = 1; k < nsq; ++k) sq[nsq + k] = 1.0 / std::sqrt((double)k);
  return cudaMemcpy(w.sqrt_tab, sq.data(), sq.size() * sizeof(double), cudaMemcpyHostToDevice);
}

cudaError_t delta_setup(DeltaWork& w, int L, int device, int method) {
  return method == kDeltaRisbo ? risbo_setup(w, L, device) : column_setup(w, L, device);
}

void delta_free(DeltaWork& w) {
  void* ptrs[] = {w.table, w.slab[0], w.slab[1], w.sqrt_tab, w.barrier, w.status, w.part, w.tasks};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  w.part = nullptr;
  w.tasks = nullptr;
  w.table = w.slab[0] = w.slab[1] = w.sqrt_tab = nullptr;
  w.barrier = nullptr;
  w.status = nullptr;
}

cudaError_t delta_run(const DeltaWork& w, int L, cudaStream_t st, long long wait_ns) {
  if (w.method != kDeltaRisbo) return column_run(w, L, st);
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.barrier, 0, (4 + (size_t)w.blocks) * sizeof(unsigned int), st)) != cudaSuccess) return e;
  RisboParams P;
  P.L = L;
  P.table = w.table;
  P.slab0 = w.slab[0];
  P.slab1 = w.slab[1];
  P.sq = w.sqrt_tab;
  P.rsq = w.sqrt_tab + (2 * (size_t)L + 4);
  P.counter = w.barrier;
  P.status = w.status;
  P.part = w.part;
  P.limit_ns = wait_ns > 0 ? wait_ns : kDefaultWaitNs;
  long long cap = w.cap;
  void* args[] = {&P, &cap};
  return cudaLaunchCooperativeKernel((void*)risbo_kernel, dim3(w.blocks), dim3(w.threads), args, w.smem, st);
}

cudaError_t delta_spin_column(const double* table, int L, int s, double* U, float* Uf, cudaStream_t st) {
  const long long n = tri_ll(L);
  const int threads = 256;
  spin_column_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(table, L, s, U, Uf);
  return cudaGetLastError();
}

}  // namespace ssht

// ---------------------------------------------------------------------------------------------
// Entry point that allocates no device memory (ssht_wigner_delta_noalloc).
//
// Some callers cannot call cudaMalloc: a host application may have reserved nearly all device
// memory for its own pool before loading this library, or the caller may run in a latency-
// critical loop where an allocation (and the device-wide synchronisation cudaMalloc/cudaFree
// can cause) is not acceptable.  For them the recursion's scratch -- the two octant slabs, the
// square-root tables, the grid-barrier words and the status word -- lives in the file-scope
// array below, sized for band-limits up to kNoAllocMaxL.  Every GPU that loads this library
// holds the array (about 2.1 MB) until the process exits.
// ---------------------------------------------------------------------------------------------
namespace ssht {
namespace {

constexpr int kNoAllocMaxL = 512;
// doubles: two padded octant slabs, the sqrt table and the reciprocal sqrt table (2L + 4
// entries each), then the
// synchronisation words: barrier counter, abort flag, status, one spare, and one degree flag
// per CTA (at most kNoAllocMaxCtas CTAs, one per SM).
constexpr size_t kNoAllocSlab = slab_doubles(kNoAllocMaxL);
constexpr size_t kNoAllocSqrt = 2 * (size_t)kNoAllocMaxL + 4;
constexpr int kNoAllocMaxCtas = 1024;
constexpr size_t kNoAllocWordDoubles = (4 + kNoAllocMaxCtas) / 2;
constexpr size_t kNoAllocDoubles = 2 * kNoAllocSlab + 2 * kNoAllocSqrt + kNoAllocWordDoubles;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// sq[k] = sqrt(k) and sq[n + k] = 1/sqrt(k) (0 for k = 0), k < n: the values the host tables
// of delta_setup hold (both are correctly rounded operations).
__global__ void noalloc_sqrt_kernel(double* sq, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    const double r = sqrt((double)k);
    sq[k] = r;
    sq[n + k] = k > 0 ? 1.0 / r : 0.0;
  }
}

// Marks an incomplete table: a barrier timeout leaves NaN in out[0] (normally Delta^0_00 = 1).
__global__ void noalloc_finish_kernel(const int* status, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *status != 0) out[0] = __longlong_as_double(0x7ff8000000000000ll);
}

std::mutex g_noalloc_mutex;
std::atomic<long long> g_noalloc_limit_ns{0};  // test hook: the entry point's spin limit (0: the default)

struct NoAllocDevice {
  double* base = nullptr;  // device address of g_noalloc_scratch on this device
  bool ready = false;
};
constexpr int kMaxDevices = 64;
NoAllocDevice g_noalloc_dev[kMaxDevices];

}  // namespace
}  // namespace ssht

extern "C" int ssht_wigner_delta_noalloc(int L, double* out, void* stream) {
  using namespace ssht;
  if (L < 1 || L > kNoAllocMaxL)
    return set_last_error(SSHT_EINVAL, "ssht_wigner_delta_noalloc: L must be in [1, 512] (the size of its fixed scratch)");
  if (!out) return set_last_error(SSHT_EINVAL, "ssht_wigner_delta_noalloc: null output");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_last_error(SSHT_ECUDA, "ssht_wigner_delta_noalloc: no usable current device");
  cudaStream_t st = (cudaStream_t)stream;
  NoAllocDevice& d = g_noalloc_dev[dev];
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  auto cuda_fail = [](const char* what, cudaError_t e) {
    return set_last_error(SSHT_ECUDA, (std::string("ssht_wigner_delta_noalloc: ") + what + ": " +
                                       cudaGetErrorString(e)).c_str());
  };
  cudaError_t ce;
  if (!d.ready) {
    // The set-up fills the square-root table with a kernel and waits for it, so it must not be
    // recorded into a graph (the fill would then only happen at the graph's launch).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((ce = cudaStreamIsCapturing(st, &cs)) != cudaSuccess) return cuda_fail("cudaStreamIsCapturing", ce);
    if (cs != cudaStreamCaptureStatusNone)
      return set_last_error(SSHT_EINVAL, "ssht_wigner_delta_noalloc: the first call on a device sets the device up and "
                                         "must not be made during stream capture");
    // Once per device, with that device current: the device address of the scratch array.
    void* p = nullptr;
    if ((ce = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return cuda_fail("cudaGetSymbolAddress", ce);
    d.base = (double*)p;
    int smem_optin = 0, per_sm = 0;
    if ((ce = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
      return cuda_fail("shared-memory attribute query", ce);
    const size_t smem = (size_t)std::min(smem_optin - 1024, 200 * 1024);
    if ((ce = cudaFuncSetAttribute(risbo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return cuda_fail("cudaFuncSetAttribute", ce);
    if ((ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, risbo_kernel, kThreads, smem)) != cudaSuccess)
      return cuda_fail("occupancy query", ce);
    if (per_sm < 1)
      return set_last_error(SSHT_ECUDA, "ssht_wigner_delta_noalloc: the recursion kernel does not fit on an SM");
    double* sq = d.base + 2 * kNoAllocSlab;
    noalloc_sqrt_kernel<<<(unsigned)((kNoAllocSqrt + 255) / 256), 256, 0, st>>>(sq, (int)kNoAllocSqrt);
    if ((ce = cudaGetLastError()) != cudaSuccess) return cuda_fail("square-root table launch", ce);
    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail("square-root table", ce);
    d.ready = true;
  }
  int sms = 0, smem_optin = 0;
  if ((ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail("SM count query", ce);
  if ((ce = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return cuda_fail("shared-memory attribute query", ce);
  const size_t smem = (size_t)std::min(smem_optin - 1024, 200 * 1024);
  if (sms > kNoAllocMaxCtas)
    return set_last_error(SSHT_EUNSUPPORTED, "ssht_wigner_delta_noalloc: more SMs than its fixed scratch has flags for");
  unsigned int* words = (unsigned int*)(d.base + 2 * kNoAllocSlab + 2 * kNoAllocSqrt);  // counter, abort, status, -, flags
  // The array keeps the previous call's contents: the synchronisation words start at zero.
  if ((ce = cudaMemsetAsync(words, 0, (4 + (size_t)sms) * sizeof(unsigned int), st)) != cudaSuccess)
    return cuda_fail("synchronisation-word reset", ce);
  RisboParams P;
  P.L = L;
  P.table = out;
  P.slab0 = d.base;
  P.slab1 = d.base + kNoAllocSlab;
  P.sq = d.base + 2 * kNoAllocSlab;
  P.rsq = P.sq + kNoAllocSqrt;
  P.counter = words;
  P.status = (int*)(words + 2);
  P.part = nullptr;  // no table: the kernel computes each step's partition
  const long long lim = g_noalloc_limit_ns.load();
  P.limit_ns = lim > 0 ? lim : kDefaultWaitNs;
  long long cap = (long long)((smem - sq_smem_bytes(L)) / sizeof(double));  // the chunk area, then the sqrt table
  void* args[] = {&P, &cap};
  if (cudaLaunchCooperativeKernel((void*)risbo_kernel, dim3(sms), dim3(kThreads), args, smem, st) != cudaSuccess)
    return set_last_error(SSHT_ECUDA, "ssht_wigner_delta_noalloc: recursion launch failed");
  noalloc_finish_kernel<<<1, 32, 0, st>>>(P.status, out);
  if (cudaGetLastError() != cudaSuccess) return set_last_error(SSHT_ECUDA, "ssht_wigner_delta_noalloc: launch failed");
  return SSHT_OK;
}

extern "C" int ssht_debug_noalloc_wait_limit(long long ns) {
  using namespace ssht;
  if (ns < 0) return set_last_error(SSHT_EINVAL, "ssht_debug_noalloc_wait_limit: ns must be >= 0");
  g_noalloc_limit_ns.store(ns);
  return SSHT_OK;
}
