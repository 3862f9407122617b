// The O(L^3) contractions on CUDA cores, FP64 (and FP32 data with the same code).
//
// Inverse (eqn fourier_coeff, Sec. 3.1), for m' >= 0:
//   F_{m m'} = (-1)^s i^{-(m+s)} sum_{l >= max(|m|, m', |s|)} U_l[m'] Delta^l_{m' m} sf_lm,
//   U_l[m'] = sqrt((2l+1)/4pi) Delta^l_{m',-s}.
// One thread owns (|m|, m') and computes F for +m and -m together, using
// Delta^l_{m',-m} = (-1)^{l+m'} Delta^l_{m' m} (eqn wignerd_sym6): one product U * Delta per
// degree serves both signs of m and every field of the thread.  The result is written as the
// input of the theta synthesis: F_{m m'} e^{i pi m'/N} at k = m' and, by eqn Ffourier_sym,
// (-1)^{m+s} F_{m m'} e^{-i pi m'/N} at k = N - m' (the phase of eqn idft_spatial).
//
// Projection (forward transform and adjoint), for l >= |s|:
//   sf_lm = (-1)^s i^{m+s} sum_{m'=0}^{l} U_l[m'] Delta^l_{m' m} H_{m m'}
// where H already folds the m' < 0 half (H_{m m'} = G_{m m'} + (-1)^{m+s} G_{m,-m'}).  One warp
// owns (l, |m|); the lanes stride over m' and the sums are closed with warp shuffles.  Rows
// of the quadrant table are read contiguously through Delta^l_{m' m} = (-1)^{m'-m} Delta^l_{m m'}.
#include "ssht_internal.h"
#include "bounds.cuh"

namespace ssht {
namespace {

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

__host__ __device__ __forceinline__ long long tri_ll(long long m) { return m * (m + 1) / 2; }
__host__ __device__ __forceinline__ size_t doff(long long l) { return (size_t)(l * (l + 1) * (2 * l + 1) / 6); }

// (re, im) of (-1)^s i^{k}
__device__ __forceinline__ void phase_ik(int s, int k, double* re, double* im) {
  const int r = ((k % 4) + 4) % 4;
  double a = (r == 0) ? 1.0 : (r == 2) ? -1.0 : 0.0;
  double b = (r == 1) ? 1.0 : (r == 3) ? -1.0 : 0.0;
  if (s & 1) { a = -a; b = -b; }
  *re = a;
  *im = b;
}

template <typename T, int BB>
__global__ void __launch_bounds__(256) inverse_kernel(int L, int s, int B, const double* __restrict__ table,
                                                      const double* __restrict__ U,
                                                      const typename Cplx<T>::type* __restrict__ flm,
                                                      typename Cplx<T>::type* __restrict__ E,
                                                      const double2* __restrict__ ph, int half, long long in_n,
                                                      long long out_n) {
  using C = typename Cplx<T>::type;
  const int Lp = L - 1, N = 2 * L - 1;
  const int m = blockIdx.x * 32 + threadIdx.x;  // |m|
  const int mp = blockIdx.y * 8 + threadIdx.y;  // m'
  const int b0 = blockIdx.z * BB;
  if (m > Lp || mp > Lp) return;
  const int as = s < 0 ? -s : s;
  int lmin = m > mp ? m : mp;
  if (lmin < as) lmin = as;
  T pr[BB], pi[BB], ner[BB], nei[BB], nor[BB], noi[BB];
#pragma unroll
  for (int j = 0; j < BB; ++j) { pr[j] = pi[j] = ner[j] = nei[j] = nor[j] = noi[j] = T(0); }
  for (int l = lmin; l <= Lp; ++l) {
    const T t = (T)(U[tri_ll(l) + mp] * table[doff(l) + (size_t)mp * (l + 1) + m]);
    const size_t cp = (size_t)l * l + l + m, cn = (size_t)l * l + l - m;
#pragma unroll
    for (int j = 0; j < BB; ++j) {
      if (b0 + j < B) {
        const long long fb = (long long)(b0 + j) * L * L;
        C a, an;
        a.x = a.y = an.x = an.y = T(0);
        if (in_bounds(fb + (long long)cp, in_n, kbSimtIn)) a = flm[fb + cp];
        if (in_bounds(fb + (long long)cn, in_n, kbSimtIn)) an = flm[fb + cn];
        pr[j] = fma(t, (T)a.x, pr[j]);
        pi[j] = fma(t, (T)a.y, pi[j]);
        if (l & 1) {
          nor[j] = fma(t, (T)an.x, nor[j]);
          noi[j] = fma(t, (T)an.y, noi[j]);
        } else {
          ner[j] = fma(t, (T)an.x, ner[j]);
          nei[j] = fma(t, (T)an.y, nei[j]);
        }
      }
    }
  }
  // phases: F_{m m'} = (-1)^s i^{-(m+s)} acc; theta phase e^{+/- i pi m'/N}
  const double2 eth = ph[(N - 1) + mp];   // e^{i pi m'/N}
  const double2 ethc = ph[(N - 1) - mp];  // e^{-i pi m'/N}
  for (int sgn = 0; sgn < 2; ++sgn) {
    if (sgn == 1 && m == 0) break;
    const int mm = sgn ? -m : m;
    double fr, fi;
    phase_ik(s, -(mm + s), &fr, &fi);
    const double sig = ((mm + s) & 1) ? -1.0 : 1.0;  // (-1)^{m+s}
    const double msign = (sgn == 1 && (mp & 1)) ? -1.0 : 1.0;  // (-1)^{m'} for -m
#pragma unroll
    for (int j = 0; j < BB; ++j) {
      if (b0 + j >= B) continue;
      double ar, ai;
      if (sgn == 0) { ar = pr[j]; ai = pi[j]; }
      else { ar = msign * ((double)ner[j] - (double)nor[j]); ai = msign * ((double)nei[j] - (double)noi[j]); }
      const double Fr = fr * ar - fi * ai, Fi = fr * ai + fi * ar;
      C v;
      if (half) {
        v.x = (T)Fr;
        v.y = (T)Fi;
        const long long o = ((long long)(b0 + j) * N + (mm + Lp)) * L + mp;
        if (in_bounds(o, out_n, kbSimtOut)) E[o] = v;
        continue;
      }
      C* row = E + ((size_t)(b0 + j) * N + (mm + Lp)) * N;
      v.x = (T)(Fr * eth.x - Fi * eth.y);
      v.y = (T)(Fr * eth.y + Fi * eth.x);
      const long long o = ((long long)(b0 + j) * N + (mm + Lp)) * N;
      if (in_bounds(o + mp, out_n, kbSimtOut)) row[mp] = v;
      if (mp > 0) {
        v.x = (T)(sig * (Fr * ethc.x - Fi * ethc.y));
        v.y = (T)(sig * (Fr * ethc.y + Fi * ethc.x));
        if (in_bounds(o + N - mp, out_n, kbSimtOut)) row[N - mp] = v;
      }
    }
  }
}

template <typename T, int BB>
__global__ void __launch_bounds__(256) project_kernel(int L, int s, int B, const double* __restrict__ table,
                                                      const double* __restrict__ U,
                                                      const typename Cplx<T>::type* __restrict__ H,
                                                      typename Cplx<T>::type* __restrict__ flm, long long in_n,
                                                      long long out_n) {
  using C = typename Cplx<T>::type;
  const int Lp = L - 1;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= tri_ll(L)) return;
  int l = (int)((sqrt(8.0 * (double)warp + 1.0) - 1.0) * 0.5);
  while (l > 0 && tri_ll(l) > warp) --l;
  while (tri_ll(l + 1) <= warp) ++l;
  const int m = (int)(warp - tri_ll(l));  // |m| <= l
  const int b0 = blockIdx.y * BB;
  T ppr[BB], ppi[BB], npr[BB], npi[BB];
#pragma unroll
  for (int j = 0; j < BB; ++j) { ppr[j] = ppi[j] = npr[j] = npi[j] = T(0); }
  const double* Trow = table + doff(l) + (size_t)m * (l + 1);  // Delta^l_{m, m'}
  const double* Ul = U + tri_ll(l);
  const int N = 2 * L - 1;
  for (int mp = lane; mp <= l; mp += 32) {
    const T v = (T)(Trow[mp] * Ul[mp]);
#pragma unroll
    for (int j = 0; j < BB; ++j) {
      if (b0 + j < B) {
        const long long ip = ((long long)(b0 + j) * N + (m + Lp)) * L + mp, in = ((long long)(b0 + j) * N + (Lp - m)) * L + mp;
        C hp, hn;
        hp.x = hp.y = hn.x = hn.y = T(0);
        if (in_bounds(ip, in_n, kbSimtIn)) hp = H[ip];
        if (in_bounds(in, in_n, kbSimtIn)) hn = H[in];
        ppr[j] = fma(v, (T)hp.x, ppr[j]);
        ppi[j] = fma(v, (T)hp.y, ppi[j]);
        npr[j] = fma(v, (T)hn.x, npr[j]);
        npi[j] = fma(v, (T)hn.y, npi[j]);
      }
    }
  }
  // the (-1)^{m'} of the +m sum follows the lane parity (m' = lane mod 32 is even/odd with lane)
  const T lsign = (lane & 1) ? T(-1) : T(1);
#pragma unroll
  for (int j = 0; j < BB; ++j) {
    ppr[j] *= lsign;
    ppi[j] *= lsign;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ppr[j] += __shfl_xor_sync(0xffffffffu, ppr[j], o);
      ppi[j] += __shfl_xor_sync(0xffffffffu, ppi[j], o);
      npr[j] += __shfl_xor_sync(0xffffffffu, npr[j], o);
      npi[j] += __shfl_xor_sync(0xffffffffu, npi[j], o);
    }
  }
  if (lane != 0) return;
  for (int sgn = 0; sgn < 2; ++sgn) {
    if (sgn == 1 && m == 0) break;
    const int mm = sgn ? -m : m;
    double fr, fi;
    phase_ik(s, mm + s, &fr, &fi);
    // +m: (-1)^m; -m: (-1)^{l+m}
    const double sg = sgn ? (((l + m) & 1) ? -1.0 : 1.0) : ((m & 1) ? -1.0 : 1.0);
#pragma unroll
    for (int j = 0; j < BB; ++j) {
      if (b0 + j >= B) continue;
      const double ar = sg * (double)(sgn ? npr[j] : ppr[j]);
      const double ai = sg * (double)(sgn ? npi[j] : ppi[j]);
      C out;
      out.x = (T)(fr * ar - fi * ai);
      out.y = (T)(fr * ai + fi * ar);
      const long long o = (long long)(b0 + j) * L * L + (long long)l * l + l + mm;
      if (in_bounds(o, out_n, kbSimtOut)) flm[o] = out;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t contract_inverse_simt(const Dims& d, int s, int B, const double* table, const double* U,
                                  const void* flm, size_t flm_bytes, void* E, size_t e_bytes, const double2* ph, int half,
                                  cudaStream_t st) {
  using C = typename Cplx<T>::type;
  constexpr int BB = 2;
  dim3 block(32, 8);
  dim3 grid((d.L + 31) / 32, (d.L + 7) / 8, (B + BB - 1) / BB);
  inverse_kernel<T, BB><<<grid, block, 0, st>>>(d.L, s, B, table, U, (const C*)flm, (C*)E, ph, half,
                                                    (long long)(flm_bytes / sizeof(C)), (long long)(e_bytes / sizeof(C)));
  return cudaGetLastError();
}

template <typename T>
cudaError_t contract_project_simt(const Dims& d, int s, int B, const double* table, const double* U,
                                  const void* H, size_t h_bytes, void* flm, size_t flm_bytes, cudaStream_t st) {
  using C = typename Cplx<T>::type;
  constexpr int BB = 2;
  const long long warps = tri_ll(d.L);
  const int threads = 256;
  dim3 grid((unsigned)((warps * 32 + threads - 1) / threads), (B + BB - 1) / BB);
  project_kernel<T, BB><<<grid, threads, 0, st>>>(d.L, s, B, table, U, (const C*)H, (C*)flm, (long long)(h_bytes / sizeof(C)),
                                                   (long long)(flm_bytes / sizeof(C)));
  return cudaGetLastError();
}

template cudaError_t contract_inverse_simt<double>(const Dims&, int, int, const double*, const double*, const void*, size_t, void*,
                                                   size_t, const double2*, int, cudaStream_t);
template cudaError_t contract_inverse_simt<float>(const Dims&, int, int, const double*, const double*, const void*, size_t, void*,
                                                  size_t, const double2*, int, cudaStream_t);
template cudaError_t contract_project_simt<double>(const Dims&, int, int, const double*, const double*, const void*, size_t, void*,
                                                   size_t, cudaStream_t);
template cudaError_t contract_project_simt<float>(const Dims&, int, int, const double*, const double*, const void*, size_t, void*,
                                                  size_t, cudaStream_t);

SSHT_BOUNDS_TU(contract_simt)

}  // namespace ssht
