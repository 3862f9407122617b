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
// Storage.  Integer degree l: octant slab Y[m(m+1)/2 + n], 0 <= n <= m <= l.
// Half-integer degree l+1/2: rows a = A + 1/2 (A = 0..l), columns b = B - 1/2 (B = 0..A+1),
// i.e. the octant plus the column b = -1/2, at A(A+3)/2 + B.
//
// Parallel layout.  One cooperative persistent grid walks l.  For the step l -> l+1 the
// rows of the new integer slab are split over the CTAs by equal entry counts.  A CTA that
// owns integer rows [r0, r1) works through them in chunks [c0, c1) sized to its shared
// memory: it copies the contiguous packed integer rows [c0-1, c1] of degree l from global
// memory into shared memory (coalesced), computes from them the half-integer rows
// [c0-1, c1-1] (one row is also computed by the neighbouring chunk), then the integer rows
// [c0, c1), which it writes to the next octant buffer and, in both orientations, to the
// quadrant table.  So each degree costs one grid barrier, and the four operands of every
// update come from shared memory.  The barrier spins at most one second, then latches a
// status bit and every CTA leaves the kernel.
#include "ssht_internal.h"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

namespace ssht {
namespace {

#ifndef SSHT_RISBO_THREADS
#define SSHT_RISBO_THREADS 512
#endif
#ifndef SSHT_RISBO_UNROLL
#define SSHT_RISBO_UNROLL 1
#endif
#ifndef SSHT_RISBO_MARK
#define SSHT_RISBO_MARK(k)  // phase boundary: 1 prologue, 2 staged, 3 half step, 4 integer step, 5 barrier
#endif
constexpr int kThreads = SSHT_RISBO_THREADS;

struct RisboParams {
  int L;
  double* table;
  double* slab0;
  double* slab1;
  const double* sq;         // sqrt(k)
  unsigned int* counter;    // [0] barrier counter, [1] abort flag (reset before launch)
  int* status;              // latched status bits
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
__device__ bool grid_barrier(unsigned int* counter, unsigned int target, int* status, Side side) {
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
        if (globaltimer_ns() - t0 > 1000000000ull) {
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
__host__ __device__ __forceinline__ long long hoff_ll(long long A) { return A * (A + 3) / 2; }

// Largest m with tri(m) <= e.
__device__ __forceinline__ int tri_row(long long e) {
  int m = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (m > 0 && tri_ll(m) > e) --m;
  while (tri_ll(m + 1) <= e) ++m;
  return m;
}

// Largest A with hoff(A) <= i.
__device__ __forceinline__ int hoff_row(long long i) {
  int A = (int)((sqrtf(8.0f * (float)i + 9.0f) - 3.0f) * 0.5f);
  if (A < 0) A = 0;
  while (A > 0 && hoff_ll(A) > i) --A;
  while (hoff_ll(A + 1) <= i) ++A;
  return A;
}

// Work of integer rows [0, m) of a step, half rows included: row m costs (m+1) integer and
// (m+2) half-integer updates, so C(m) = sum_{k<m} (2k+3) = m^2 + 2m.
__host__ __device__ __forceinline__ long long row_cost(long long m) { return m * m + 2 * m; }

// Smallest m with C(m) >= x.  FP32 first guess, exact integer correction (FP64 arithmetic is
// costly on this part and is kept for the recursion itself).
__host__ __device__ __forceinline__ int share_row(long long x, int rows) {
  int m = (int)(sqrtf(1.0f + (float)x) - 1.0f);
  if (m < 0) m = 0;
  if (m > rows) m = rows;
  while (m > 0 && row_cost(m - 1) >= x) --m;
  while (m < rows && row_cost(m) < x) ++m;
  return m;
}

// Rows [r0, r1) of the new integer slab of degree lp owned by CTA cta of nb, balanced on C.
__host__ __device__ __forceinline__ void cta_rows(int lp, int cta, int nb, int* r0, int* r1) {
  const long long S = row_cost(lp + 1);
  *r0 = share_row(S * cta / nb, lp + 1);
  *r1 = share_row(S * (cta + 1) / nb, lp + 1);
}

// v with its sign flipped when neg is set, by integer ops on the sign bit (a multiplication by
// -1 would cost an FP64 instruction).
__device__ __forceinline__ double flip(double v, bool neg) {
  return __hiloint2double(__double2hiint(v) ^ (neg ? (int)0x80000000 : 0), __double2loint(v));
}

// Integer slab of degree l staged in shared memory from row ybase on (packed rows), any (m, n)
// with 0 <= m <= l+1 and -1 <= n <= m+1.
__device__ __forceinline__ double yget(const double* __restrict__ Y, int l, long long ybase, int m, int n) {
  bool neg = false;
  if (n == -1) {
    if (m == 0) {  // Delta_{0,-1} = (-1)^l Delta_{0,1} = (-1)^{l+1} Delta_{1,0}
      neg = (l & 1) == 0;
      m = 1;
      n = 0;
    } else {       // Delta_{m,-1} = (-1)^{l+m} Delta_{m,1}
      neg = ((l + m) & 1) != 0;
      n = 1;
    }
  }
  if (n > m) {     // transpose
    if ((n - m) & 1) neg = !neg;
    const int t = m; m = n; n = t;
  }
  if (m > l) return 0.0;
  return flip(Y[tri_ll(m) + n - ybase], neg);
}

// Half-integer slab of degree l+1/2 held in shared memory from row Alo on,
// any (A, B) with -1 <= A <= l+1 and 0 <= B <= A+2.
__device__ __forceinline__ double xget(const double* __restrict__ X, int l, long long hbase, int A, int B) {
  bool neg = false;
  if (A == -1) {   // a = -1/2
    if (B == 0) {  // (-1/2,-1/2) = (1/2,1/2)
      A = 0; B = 1;
    } else {       // (-1/2,1/2) = -(1/2,-1/2)
      A = 0; B = 0; neg = true;
    }
  }
  if (B > A + 1) { // b > a: transpose (a,b) -> (b,a), sign (-1)^{a-b}
    if ((B - A - 1) & 1) neg = !neg;
    const int nA = B - 1, nB = A + 1;
    A = nA; B = nB;
  }
  if (A > l) return 0.0;
  return flip(X[hoff_ll(A) + B - hbase], neg);
}

// Shared-memory doubles needed to produce integer rows [c0, c1) of degree l+1 from degree l:
// the staged integer rows [Alo, min(Ahi+1, l)] and the half rows [Alo, Ahi].
__host__ __device__ __forceinline__ long long chunk_need(int l, int c0, int c1) {
  const int Alo = c0 > 0 ? c0 - 1 : 0;
  const int Ahi = (c1 - 1 < l) ? c1 - 1 : l;
  const int Ytop = (Ahi + 1 < l) ? Ahi + 1 : l;
  return (tri_ll(Ytop + 1) - tri_ll(Alo)) + (hoff_ll(Ahi + 1) - hoff_ll(Alo));
}

// 1/k to FP64 accuracy without an FP64 division: FP32 reciprocal, then two Newton steps.
__device__ __forceinline__ double recip(double k) {
  double r = (double)(1.0f / (float)k);
  r = r * fma(-k, r, 2.0);
  r = r * fma(-k, r, 2.0);
  return r;
}

constexpr int kUnroll = SSHT_RISBO_UNROLL;  // independent updates in flight per thread
constexpr int kRowCap = 512; // rows of pre-scaled row factors kept per chunk

__global__ void __launch_bounds__(kThreads, 1) risbo_kernel(RisboParams P, long long cap) {
  extern __shared__ double smem[];
  __shared__ int s_rows[2];
  __shared__ double s_scale[2];
  // Rows and step scales p/(2j) of step l -> l + 1, computed while the previous barrier waits.
  auto params = [&](int l) {
    const int lp = l + 1;
    cta_rows(lp, blockIdx.x, gridDim.x, &s_rows[0], &s_rows[1]);
    s_scale[0] = 0.70710678118654752440 * recip((double)(2 * l + 1));
    s_scale[1] = 0.70710678118654752440 * recip((double)(2 * lp));
  };
  // row factors sqrt(j+a) p/(2j), sqrt(j-a) p/(2j) of the half step (s_ra, s_rb) and the integer step
  __shared__ double s_ra[kRowCap + 2], s_rb[kRowCap + 2], s_ia[kRowCap + 2], s_ib[kRowCap + 2];
  const int nb = gridDim.x;
  const int cta = blockIdx.x;
  if (cta == 0 && threadIdx.x == 0) {
    P.slab0[0] = 1.0;
    P.table[0] = 1.0;
  }
  unsigned int phase = 1;
  if (!grid_barrier(P.counter, phase * nb, P.status, [&] { params(0); })) return;
  for (int l = 0; l + 1 < P.L; ++l) {
    const double* __restrict__ Yg = (l & 1) ? P.slab1 : P.slab0;
    double* __restrict__ Yn = (l & 1) ? P.slab0 : P.slab1;
    const int lp = l + 1;
    const int r0 = s_rows[0], r1 = s_rows[1];
    const double sc = s_scale[0], sc2 = s_scale[1];
    SSHT_RISBO_MARK(1);
    double* __restrict__ T = P.table + (size_t)((long long)lp * (lp + 1) * (2 * lp + 1) / 6);
    for (int c0 = r0; c0 < r1;) {
      // Largest c1 <= min(r1, c0 + kRowCap) whose chunk fits (chunk_need grows with c1).
      int lo = c0 + 1, hi = (r1 < c0 + kRowCap) ? r1 : c0 + kRowCap;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunk_need(l, c0, mid) <= cap) lo = mid; else hi = mid - 1;
      }
      const int c1 = lo;
      const int Alo = c0 > 0 ? c0 - 1 : 0;
      const int Ahi = (c1 - 1 < l) ? c1 - 1 : l;
      const int Ytop = (Ahi + 1 < l) ? Ahi + 1 : l;
      const long long ybase = tri_ll(Alo);
      const int ycount = (int)(tri_ll(Ytop + 1) - ybase);
      const long long hbase = hoff_ll(Alo);
      const int hcount = (int)(hoff_ll(Ahi + 1) - hbase);
      double* __restrict__ Ys = smem;
      double* __restrict__ Xs = smem + ycount;
      __syncthreads();  // the previous chunk is done with shared memory
      // Stage the contiguous packed rows [Alo, Ytop] of the integer slab (asynchronous copies,
      // all in flight together); pre-scale the row factors meanwhile.
      for (int i = threadIdx.x; i < ycount; i += blockDim.x) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(Ys + i);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(Yg + ybase + i) : "memory");
      }
      for (int A = Alo + (int)threadIdx.x; A <= Ahi; A += blockDim.x) {
        s_ra[A - Alo] = P.sq[l + A + 1] * sc;  // j + a = l + A + 1
        s_rb[A - Alo] = P.sq[l - A] * sc;      // j - a = l - A
      }
      for (int m = c0 + (int)threadIdx.x; m < c1; m += blockDim.x) {
        s_ia[m - c0] = P.sq[lp + m] * sc2;
        s_ib[m - c0] = P.sq[lp - m] * sc2;
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      SSHT_RISBO_MARK(2);
      // Half step l -> l + 1/2 (2j = 2l + 1): j+b = l+B, j-b = l+1-B.
      for (int base = threadIdx.x; base < hcount; base += kUnroll * blockDim.x) {
        double x1[kUnroll], x2[kUnroll], x3[kUnroll], x4[kUnroll], sb[kUnroll], smb[kUnroll], ra[kUnroll], rb[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int i = base + u * blockDim.x;
          const int ii = i < hcount ? i : hcount - 1;
          const int A = hoff_row(hbase + ii);
          const int B = (int)(hbase + ii - hoff_ll(A));
          x1[u] = yget(Ys, l, ybase, A, B - 1);
          x2[u] = yget(Ys, l, ybase, A, B);
          x3[u] = yget(Ys, l, ybase, A + 1, B - 1);
          x4[u] = yget(Ys, l, ybase, A + 1, B);
          sb[u] = P.sq[l + B];
          smb[u] = P.sq[l + 1 - B];
          ra[u] = s_ra[A - Alo];
          rb[u] = s_rb[A - Alo];
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int i = base + u * blockDim.x;
          const double t1 = fma(-smb[u], x2[u], sb[u] * x1[u]);
          const double t2 = fma(smb[u], x4[u], sb[u] * x3[u]);
          const double v = fma(ra[u], t1, rb[u] * t2);
          if (i < hcount) Xs[i] = v;
        }
      }
      __syncthreads();
      SSHT_RISBO_MARK(3);
      // Integer step l + 1/2 -> lp (2j = 2 lp).
      const long long e0 = tri_ll(c0);
      const int ecount = (int)(tri_ll(c1) - e0);
      for (int base = threadIdx.x; base < ecount; base += kUnroll * blockDim.x) {
        double x1[kUnroll], x2[kUnroll], x3[kUnroll], x4[kUnroll], sb[kUnroll], smb[kUnroll], ra[kUnroll], rb[kUnroll];
        int mm[kUnroll], nn[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int i = base + u * blockDim.x;
          const long long e = e0 + (i < ecount ? i : ecount - 1);
          const int m = tri_row(e);
          const int n = (int)(e - tri_ll(m));
          mm[u] = m;
          nn[u] = n;
          x1[u] = xget(Xs, l, hbase, m - 1, n);
          x2[u] = xget(Xs, l, hbase, m - 1, n + 1);
          x3[u] = xget(Xs, l, hbase, m, n);
          x4[u] = xget(Xs, l, hbase, m, n + 1);
          sb[u] = P.sq[lp + n];
          smb[u] = P.sq[lp - n];
          ra[u] = s_ia[m - c0];
          rb[u] = s_ib[m - c0];
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int i = base + u * blockDim.x;
          const double t1 = fma(-smb[u], x2[u], sb[u] * x1[u]);
          const double t2 = fma(smb[u], x4[u], sb[u] * x3[u]);
          const double v = fma(ra[u], t1, rb[u] * t2);
          if (i < ecount) {
            const int m = mm[u], n = nn[u];
            Yn[e0 + i] = v;
            T[(size_t)m * (lp + 1) + n] = v;
            if (n != m) T[(size_t)n * (lp + 1) + m] = flip(v, ((m - n) & 1) != 0);
          }
        }
      }
      SSHT_RISBO_MARK(4);
      c0 = c1;
    }
    ++phase;
    if (!grid_barrier(P.counter, phase * nb, P.status, [&] { params(l + 1); })) return;
    SSHT_RISBO_MARK(5);
  }
}

// U[tri(l) + m'] = sqrt((2l+1)/4pi) Delta^l_{m',-s} for l >= |s|, 0 otherwise.
__global__ void spin_column_kernel(const double* __restrict__ table, int L, int s, double* __restrict__ U) {
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
}

}  // namespace

cudaError_t delta_setup(DeltaWork& w, int L, int device) {
  cudaError_t e;
  int sms = 0, per_sm = 0, smem_optin = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess) return e;
  w.threads = kThreads;
  w.blocks = sms;  // one CTA per SM
  // Shared memory: as much as one CTA per SM may take, leaving room for the static part.
  w.smem = (size_t)std::min(smem_optin - 1024, 200 * 1024);
  w.cap = (long long)(w.smem / sizeof(double));
  // Every chunk holds at least one row: the widest single-row chunk (last degree) must fit.
  for (int m = 0; m < L; ++m)
    if (chunk_need(L - 2 > 0 ? L - 2 : 0, m, m + 1) > w.cap) return cudaErrorInvalidValue;
  if ((e = cudaFuncSetAttribute(risbo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w.smem)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, risbo_kernel, kThreads, w.smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  if ((e = cudaMalloc(&w.table, delta_offset(L) * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.slab[0], tri(L + 1) * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.slab[1], tri(L + 1) * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.sqrt_tab, (2 * (size_t)L + 4) * sizeof(double))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.barrier, 4 * sizeof(unsigned int))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&w.status, sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMemset(w.status, 0, sizeof(int))) != cudaSuccess) return e;
  std::vector<double> sq(2 * (size_t)L + 4);
  for (size_t k = 0; k < sq.size(); ++k) sq[k] = std::sqrt((double)k);
  return cudaMemcpy(w.sqrt_tab, sq.data(), sq.size() * sizeof(double), cudaMemcpyHostToDevice);
}

cudaError_t delta_run(const DeltaWork& w, int L, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.barrier, 0, 4 * sizeof(unsigned int), st)) != cudaSuccess) return e;
  RisboParams P;
  P.L = L;
  P.table = w.table;
  P.slab0 = w.slab[0];
  P.slab1 = w.slab[1];
  P.sq = w.sqrt_tab;
  P.counter = w.barrier;
  P.status = w.status;
  long long cap = w.cap;
  void* args[] = {&P, &cap};
  return cudaLaunchCooperativeKernel((void*)risbo_kernel, dim3(w.blocks), dim3(w.threads), args, w.smem, st);
}

cudaError_t delta_spin_column(const double* table, int L, int s, double* U, cudaStream_t st) {
  const long long n = tri_ll(L);
  const int threads = 256;
  spin_column_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(table, L, s, U);
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
// square-root table, the grid-barrier words and the status word -- lives in the file-scope
// array below, sized for band-limits up to kNoAllocMaxL.  Every GPU that loads this library
// holds the array (about 2.1 MB) until the process exits.
// ---------------------------------------------------------------------------------------------
namespace ssht {
namespace {

constexpr int kNoAllocMaxL = 512;
// doubles: two octant slabs of tri(kNoAllocMaxL + 1) entries and the sqrt table (2L + 4 entries),
// then 4 words for the barrier counter / abort flag and the status word.
constexpr size_t kNoAllocSlab = (size_t)(kNoAllocMaxL + 1) * (kNoAllocMaxL + 2) / 2;
constexpr size_t kNoAllocSqrt = 2 * (size_t)kNoAllocMaxL + 4;
constexpr size_t kNoAllocDoubles = 2 * kNoAllocSlab + kNoAllocSqrt + 4;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

__global__ void noalloc_sqrt_kernel(double* sq, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) sq[k] = sqrt((double)k);
}

// Marks an incomplete table: a barrier timeout leaves NaN in out[0] (normally Delta^0_00 = 1).
__global__ void noalloc_finish_kernel(const int* status, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *status != 0) out[0] = __longlong_as_double(0x7ff8000000000000ll);
}

std::mutex g_noalloc_mutex;

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
  if (!d.ready) {
    // Once per device, with that device current: the device address of the scratch array.
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess)
      return set_last_error(SSHT_ECUDA, "ssht_wigner_delta_noalloc: cudaGetSymbolAddress failed");
    d.base = (double*)p;
    int sms = 0, smem_optin = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SSHT_ECUDA;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return SSHT_ECUDA;
    const size_t smem = (size_t)std::min(smem_optin - 1024, 200 * 1024);
    if (cudaFuncSetAttribute(risbo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return SSHT_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, risbo_kernel, kThreads, smem) != cudaSuccess ||
        per_sm < 1)
      return SSHT_ECUDA;
    double* sq = d.base + 2 * kNoAllocSlab;
    noalloc_sqrt_kernel<<<(unsigned)((kNoAllocSqrt + 255) / 256), 256, 0, st>>>(sq, (int)kNoAllocSqrt);
    if (cudaGetLastError() != cudaSuccess) return SSHT_ECUDA;
    d.ready = true;
  }
  int sms = 0, smem_optin = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SSHT_ECUDA;
  if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return SSHT_ECUDA;
  const size_t smem = (size_t)std::min(smem_optin - 1024, 200 * 1024);
  unsigned int* words = (unsigned int*)(d.base + 2 * kNoAllocSlab + kNoAllocSqrt);  // counter, abort, status
  // The array keeps the previous call's contents: the barrier words and the status start at zero.
  if (cudaMemsetAsync(words, 0, 4 * sizeof(double), st) != cudaSuccess) return SSHT_ECUDA;
  RisboParams P;
  P.L = L;
  P.table = out;
  P.slab0 = d.base;
  P.slab1 = d.base + kNoAllocSlab;
  P.sq = d.base + 2 * kNoAllocSlab;
  P.counter = words;
  P.status = (int*)(words + 2);
  long long cap = (long long)(smem / sizeof(double));
  void* args[] = {&P, &cap};
  if (cudaLaunchCooperativeKernel((void*)risbo_kernel, dim3(sms), dim3(kThreads), args, smem, st) != cudaSuccess)
    return set_last_error(SSHT_ECUDA, "ssht_wigner_delta_noalloc: recursion launch failed");
  noalloc_finish_kernel<<<1, 32, 0, st>>>(P.status, out);
  if (cudaGetLastError() != cudaSuccess) return set_last_error(SSHT_ECUDA, "ssht_wigner_delta_noalloc: launch failed");
  return SSHT_OK;
}
