// Real fields of spin 0: f real, so sf_{l,-m} = (-1)^m conj(sf_lm) (the second conjugate symmetry
// of Sec. 3.3: with the theta parity already used by every plan, a factor of four over a transform
// that uses neither).  Two real fields ride in one complex field, f = f1 + i f2, whose
// coefficients are sf = sf1 + i sf2 by linearity; the transforms are the complex ones and these
// kernels only pack and unpack:
//   inverse:  sf = sf1 + i sf2  ->  f  ->  f1 = Re f, f2 = Im f
//   forward / adjoint:  f = f1 + i f2  ->  c  ->  sf1_lm = (c_lm + e_lm)/2, sf2_lm = (c_lm - e_lm)/(2i),
//             e_lm = (-1)^m conj(c_{l,-m})
// (e = sf1 - i sf2 because each of sf1, sf2 has the symmetry).  Field 2p and 2p+1 of the caller
// pair into complex field p; an odd count pairs the last field with zero.
#include "ssht_internal.h"
#include "bounds.cuh"

namespace ssht {
namespace {

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };

template <typename T>
__global__ void pack_coeffs_kernel(long long n2, long long npair, int nreal, const typename Cx<T>::type* __restrict__ flm,
                                   typename Cx<T>::type* __restrict__ rc, long long in_n, long long out_n) {
  using C = typename Cx<T>::type;
  const long long total = npair * n2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / n2, e = i - p * n2;
    C a, b;
    a.x = a.y = b.x = b.y = 0;
    if (in_bounds(2 * p * n2 + e, in_n, kbRealIn)) a = flm[2 * p * n2 + e];
    if (2 * p + 1 < nreal && in_bounds((2 * p + 1) * n2 + e, in_n, kbRealIn)) b = flm[(2 * p + 1) * n2 + e];
    C r;
    r.x = a.x - b.y;  // a + i b
    r.y = a.y + b.x;
    if (in_bounds(i, out_n, kbRealOut)) rc[i] = r;
  }
}

template <typename T>
__global__ void pack_grid_kernel(long long n2, long long npair, int nreal, const T* __restrict__ f,
                                 typename Cx<T>::type* __restrict__ rg, long long in_n, long long out_n) {
  using C = typename Cx<T>::type;
  const long long total = npair * n2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / n2, e = i - p * n2;
    C r;
    r.x = in_bounds(2 * p * n2 + e, in_n, kbRealIn) ? f[2 * p * n2 + e] : T(0);
    r.y = (2 * p + 1 < nreal && in_bounds((2 * p + 1) * n2 + e, in_n, kbRealIn)) ? f[(2 * p + 1) * n2 + e] : T(0);
    if (in_bounds(i, out_n, kbRealOut)) rg[i] = r;
  }
}

template <typename T>
__global__ void unpack_grid_kernel(long long n2, long long npair, int nreal, const typename Cx<T>::type* __restrict__ rg,
                                   T* __restrict__ f, long long in_n, long long out_n) {
  const long long total = npair * n2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / n2, e = i - p * n2;
    if (!in_bounds(i, in_n, kbRealIn)) continue;
    const auto z = rg[i];
    if (in_bounds(2 * p * n2 + e, out_n, kbRealOut)) f[2 * p * n2 + e] = z.x;
    if (2 * p + 1 < nreal && in_bounds((2 * p + 1) * n2 + e, out_n, kbRealOut)) f[(2 * p + 1) * n2 + e] = z.y;
  }
}

template <typename T>
__global__ void unpack_coeffs_kernel(int L, long long npair, int nreal, const typename Cx<T>::type* __restrict__ rc,
                                     typename Cx<T>::type* __restrict__ flm, long long in_n, long long out_n) {
  using C = typename Cx<T>::type;
  const long long n2 = (long long)L * L;
  const long long total = npair * n2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / n2, e = i - p * n2;
    int l = (int)sqrtf((float)e);  // e < 2^22: exact float, then an integer correction
    while ((long long)l * l > e) --l;
    while ((long long)(l + 1) * (l + 1) <= e) ++l;
    const int m = (int)(e - (long long)l * l - l);
    const long long di = p * n2 + (long long)l * l + l - m;
    if (!in_bounds(i, in_n, kbRealIn) || !in_bounds(di, in_n, kbRealIn)) continue;
    const C c = rc[i];
    const C d = rc[di];
    const T sg = (m & 1) ? T(-1) : T(1);
    const T ex = sg * d.x, ey = -sg * d.y;  // e = (-1)^m conj(d)
    C a, b;
    a.x = T(0.5) * (c.x + ex);
    a.y = T(0.5) * (c.y + ey);
    b.x = T(0.5) * (c.y - ey);  // (c - e) / (2i)
    b.y = -T(0.5) * (c.x - ex);
    if (in_bounds(2 * p * n2 + e, out_n, kbRealOut)) flm[2 * p * n2 + e] = a;
    if (2 * p + 1 < nreal && in_bounds((2 * p + 1) * n2 + e, out_n, kbRealOut)) flm[(2 * p + 1) * n2 + e] = b;
  }
}

// Spin pairs (SSHT_FLAG_SPIN_PAIR): the pair of fields (f, f*) of spins s and -s -- the signals the
// paper calls f_s* = f_{-s} -- has one set of coefficients determined by the other through the
// conjugate symmetry of Sec. 2.3: _{-s}f_{l,-m} = (-1)^{s+m} conj(_s f_{lm}).  So the pair's
// forward (or adjoint) is one spin-s transform followed by this expansion:
//   out[b][0][l,m] = c[b][l,m],  out[b][1][l,m] = (-1)^{s+m} conj(c[b][l,-m])   (zero for l < |s|);
// and its inverse needs the spin-s half only (gathered by pair_gather_kernel).
template <typename T>
__global__ void pair_expand_kernel(int L, int s, long long B, const typename Cx<T>::type* __restrict__ c,
                                   typename Cx<T>::type* __restrict__ out, long long in_n, long long out_n) {
  using C = typename Cx<T>::type;
  const long long n2 = (long long)L * L, total = B * n2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / n2, e = i - b * n2;
    int l = (int)sqrtf((float)e);
    while ((long long)l * l > e) --l;
    while ((long long)(l + 1) * (l + 1) <= e) ++l;
    const int m = (int)(e - (long long)l * l - l);
    const long long di = b * n2 + (long long)l * l + l - m;
    if (!in_bounds(i, in_n, kbPairIn) || !in_bounds(di, in_n, kbPairIn)) continue;
    const C d = c[di];
    const T sg = ((s + m) & 1) ? T(-1) : T(1);
    C q;
    q.x = sg * d.x;
    q.y = -sg * d.y;
    if (in_bounds(2 * b * n2 + e, out_n, kbPairOut)) out[2 * b * n2 + e] = c[i];
    if (in_bounds((2 * b + 1) * n2 + e, out_n, kbPairOut)) out[(2 * b + 1) * n2 + e] = q;
  }
}

template <typename T>
__global__ void pair_gather_kernel(long long n2, long long B, const typename Cx<T>::type* __restrict__ in,
                                   typename Cx<T>::type* __restrict__ c, long long in_n, long long out_n) {
  const long long total = B * n2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / n2, e = i - b * n2;
    if (in_bounds(2 * b * n2 + e, in_n, kbPairIn) && in_bounds(i, out_n, kbPairOut)) c[i] = in[2 * b * n2 + e];
  }
}

unsigned blocks_for(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

}  // namespace

template <typename T>
cudaError_t real_pack_coeffs(int L, int nreal, const void* flm, void* rc, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const long long n2 = (long long)L * L, np = (nreal + 1) / 2;
  pack_coeffs_kernel<T><<<blocks_for(np * n2), 256, 0, st>>>(n2, np, nreal, (const C*)flm, (C*)rc, nreal * n2, np * n2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t real_pack_grid(int L, int nreal, const void* f, void* rg, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const long long n2 = (long long)L * (2 * L - 1), np = (nreal + 1) / 2;
  pack_grid_kernel<T><<<blocks_for(np * n2), 256, 0, st>>>(n2, np, nreal, (const T*)f, (C*)rg, nreal * n2, np * n2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t real_unpack_grid(int L, int nreal, const void* rg, void* f, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const long long n2 = (long long)L * (2 * L - 1), np = (nreal + 1) / 2;
  unpack_grid_kernel<T><<<blocks_for(np * n2), 256, 0, st>>>(n2, np, nreal, (const C*)rg, (T*)f, np * n2, nreal * n2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t real_unpack_coeffs(int L, int nreal, const void* rc, void* flm, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const long long n2 = (long long)L * L, np = (nreal + 1) / 2;
  unpack_coeffs_kernel<T><<<blocks_for(np * n2), 256, 0, st>>>(L, np, nreal, (const C*)rc, (C*)flm, np * n2, nreal * n2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t pair_expand(int L, int s, int B, const void* c, void* out, cudaStream_t st) {
  using C = typename Cx<T>::type;
  pair_expand_kernel<T><<<blocks_for((long long)B * L * L), 256, 0, st>>>(L, s, B, (const C*)c, (C*)out, (long long)B * L * L, 2LL * B * L * L);
  return cudaGetLastError();
}

template <typename T>
cudaError_t pair_gather(int L, int B, const void* in, void* c, cudaStream_t st) {
  using C = typename Cx<T>::type;
  const long long n2 = (long long)L * L;
  pair_gather_kernel<T><<<blocks_for(B * n2), 256, 0, st>>>(n2, B, (const C*)in, (C*)c, 2LL * B * n2, (long long)B * n2);
  return cudaGetLastError();
}

cudaError_t real_setup() {
  cudaError_t e;
  if ((e = prefer_shared(pack_coeffs_kernel<double>)) != cudaSuccess) return e;
  if ((e = prefer_shared(pack_coeffs_kernel<float>)) != cudaSuccess) return e;
  if ((e = prefer_shared(pack_grid_kernel<double>)) != cudaSuccess) return e;
  if ((e = prefer_shared(pack_grid_kernel<float>)) != cudaSuccess) return e;
  if ((e = prefer_shared(unpack_grid_kernel<double>)) != cudaSuccess) return e;
  if ((e = prefer_shared(unpack_grid_kernel<float>)) != cudaSuccess) return e;
  if ((e = prefer_shared(unpack_coeffs_kernel<double>)) != cudaSuccess) return e;
  if ((e = prefer_shared(pair_expand_kernel<double>)) != cudaSuccess) return e;
  if ((e = prefer_shared(pair_expand_kernel<float>)) != cudaSuccess) return e;
  if ((e = prefer_shared(pair_gather_kernel<double>)) != cudaSuccess) return e;
  if ((e = prefer_shared(pair_gather_kernel<float>)) != cudaSuccess) return e;
  return prefer_shared(unpack_coeffs_kernel<float>);
}

#define SSHT_REAL_INST(T)                                                                          \
  template cudaError_t real_pack_coeffs<T>(int, int, const void*, void*, cudaStream_t);          \
  template cudaError_t real_pack_grid<T>(int, int, const void*, void*, cudaStream_t);            \
  template cudaError_t real_unpack_grid<T>(int, int, const void*, void*, cudaStream_t);          \
  template cudaError_t real_unpack_coeffs<T>(int, int, const void*, void*, cudaStream_t);        \
  template cudaError_t pair_expand<T>(int, int, int, const void*, void*, cudaStream_t);          \
  template cudaError_t pair_gather<T>(int, int, const void*, void*, cudaStream_t);
SSHT_REAL_INST(double)
SSHT_REAL_INST(float)
#undef SSHT_REAL_INST

SSHT_BOUNDS_TU(real)

}  // namespace ssht
