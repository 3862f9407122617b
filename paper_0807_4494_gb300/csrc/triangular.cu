// The paper's own forward transform (Sec. 3.4.2, eqn matrix_fwd), FP64: for each m the torus
// coefficients F_{m m'} (m' >= 0) of the extended signal are related to sf_{lm} by an upper
// triangular system
//   F_{m m'} = (-1)^s i^{-(m+s)} sum_{l >= max(m', lmin)} sqrt((2l+1)/4pi) Delta^l_{m'm} Delta^l_{m',-s} sf_{lm},
// rows and unknowns l, m' in [lmin, Lp], lmin = max(|m|, |s|) (rows below lmin are implied by the
// others), solved by back substitution from m' = Lp down.  The extension takes the parity
// (-1)^{m+s} of each column (the case split after eqn matrix_fwd), which is the torus stage of the
// quadrature forward without its weight convolution.  The paper reports that this solve loses
// accuracy as L grows (Sec. 4.2); it is provided to reproduce that behaviour next to the stable
// quadrature forward.
//
// Kernel: one CTA per (|m|, pair of fields), the columns of its right-hand side being (sign of
// m, field); Delta^l_{m',-m} = (-1)^{l+m'} Delta^l_{m'm} (eqn wignerd_sym6) lets both signs share
// the matrix.  Column-oriented substitution: when x_l is known, every row m' < l subtracts
// K[m'][l] x_l; rows are spread over the threads (coalesced table reads along m').
#include "ssht_internal.h"

namespace ssht {
namespace {

constexpr int TRI_THREADS = 512;
constexpr int TRI_ROWS = 4;   // rows per thread: L <= 2048
constexpr int TRI_FIELDS = 2; // fields per CTA

__host__ __device__ inline size_t doff3(long long l) { return (size_t)(l * (l + 1) * (2 * l + 1) / 6); }
__host__ __device__ inline long long tri3(long long l) { return l * (l + 1) / 2; }

// i^k (-1)^s as (re, im)
__device__ inline double2 ipow_s(int s, int k) {
  const int r = ((k % 4) + 4) % 4;
  double a = (r == 0) ? 1.0 : (r == 2) ? -1.0 : 0.0;
  double b = (r == 1) ? 1.0 : (r == 3) ? -1.0 : 0.0;
  if (s & 1) {
    a = -a;
    b = -b;
  }
  return make_double2(a, b);
}

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// Fk: [B][N][N], theta-DFT bins of the extended columns (row m + Lp, bin k = m' mod N), without
// the phase e^{-i pi m'/N} and the 1/N of eqn dft_spatial, which are applied here.
__global__ void __launch_bounds__(TRI_THREADS) tri_solve_kernel(int L, int s, int B, const double* __restrict__ table,
                                                                const double* __restrict__ U,
                                                                const double2* __restrict__ Fk,
                                                                const double2* __restrict__ ph, double2* __restrict__ flm) {
  constexpr int C = 2 * TRI_FIELDS;  // columns: (sign, field)
  __shared__ double2 xs[C];
  const int m = blockIdx.x;
  const int b0 = blockIdx.y * TRI_FIELDS;
  const int Lp = L - 1, N = 2 * L - 1;
  const int as = s < 0 ? -s : s;
  const int lmin = m > as ? m : as;
  if (lmin > Lp) return;
  const double invN = 1.0 / (double)N;
  // right-hand sides, divided by the column phase (-1)^s i^{-(mm+s)}
  double2 r[TRI_ROWS][C];
#pragma unroll
  for (int q = 0; q < TRI_ROWS; ++q) {
    const int mp = lmin + (int)threadIdx.x + q * TRI_THREADS;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      r[q][c] = make_double2(0.0, 0.0);
      const int sign = c / TRI_FIELDS, b = b0 + c % TRI_FIELDS;
      if (mp <= Lp && b < B && !(sign && m == 0)) {
        const int mm = sign ? -m : m;
        const double2 v = Fk[((size_t)b * N + (mm + Lp)) * N + mp];
        const double2 F = cmul(v, ph[-mp + N - 1]);
        const double2 unphase = ipow_s(s, mm + s);  // 1 / ((-1)^s i^{-(mm+s)})
        const double2 x = cmul(F, unphase);
        r[q][c] = make_double2(x.x * invN, x.y * invN);
      }
    }
  }
  for (int l = Lp; l >= lmin; --l) {
    const double* Tl = table + doff3(l) + (size_t)m * (l + 1);  // Delta^l_{m m'}, contiguous in m'
    const double* Ul = U + tri3(l);
    // the owner of row l solves it
    const int own = l - lmin;
    if ((int)threadIdx.x == own % TRI_THREADS) {
      const int q = own / TRI_THREADS;
      const double d = Ul[l] * Tl[l] * (((l - m) & 1) ? -1.0 : 1.0);  // U_l[l] Delta^l_{l m}
      const double inv = 1.0 / d;
#pragma unroll
      for (int qq = 0; qq < TRI_ROWS; ++qq) {
        if (qq != q) continue;
#pragma unroll
        for (int c = 0; c < C; ++c) xs[c] = make_double2(r[qq][c].x * inv, r[qq][c].y * inv);
      }
    }
    __syncthreads();
    double2 x[C];
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = xs[c];
    if (threadIdx.x == 0) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int sign = c / TRI_FIELDS, b = b0 + c % TRI_FIELDS;
        if (b < B && !(sign && m == 0)) flm[(size_t)b * L * L + (size_t)l * l + l + (sign ? -m : m)] = x[c];
      }
    }
    // rows m' < l: r[m'] -= U_l[m'] Delta^l_{m' m} x_l, with (-1)^{l+m'} for the -m columns
#pragma unroll
    for (int q = 0; q < TRI_ROWS; ++q) {
      const int mp = lmin + (int)threadIdx.x + q * TRI_THREADS;
      if (mp < l) {
        const double k = Ul[mp] * Tl[mp] * (((mp - m) & 1) ? -1.0 : 1.0);
        const double kn = ((l + mp) & 1) ? -k : k;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const double kk = (c / TRI_FIELDS) ? kn : k;
          r[q][c].x = fma(-kk, x[c].x, r[q][c].x);
          r[q][c].y = fma(-kk, x[c].y, r[q][c].y);
        }
      }
    }
    __syncthreads();
  }
}

// Coefficients with l < |s| do not exist: zero them (the solve writes l >= lmin only).
__global__ void zero_low_kernel(int L, int s, int B, double2* __restrict__ flm) {
  const int as = s < 0 ? -s : s;
  const long long n = (long long)B * as * as;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / ((long long)as * as), e = i % ((long long)as * as);
    flm[b * L * L + e] = make_double2(0.0, 0.0);
  }
}

}  // namespace

cudaError_t triangular_solve(const Dims& d, int s, int B, const double* table, const double* U, const void* Fk,
                             const double2* ph, void* flm, cudaStream_t st) {
  if (d.L > TRI_ROWS * TRI_THREADS) return cudaErrorInvalidValue;
  const int as = s < 0 ? -s : s;
  if (as > 0) {
    zero_low_kernel<<<64, 256, 0, st>>>(d.L, s, B, (double2*)flm);
  }
  dim3 grid(d.L, (B + TRI_FIELDS - 1) / TRI_FIELDS);
  tri_solve_kernel<<<grid, TRI_THREADS, 0, st>>>(d.L, s, B, table, U, (const double2*)Fk, ph, (double2*)flm);
  return cudaGetLastError();
}

}  // namespace ssht
