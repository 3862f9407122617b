// Torus-side kernels around the FFTs (Secs. 3.2 and 3.4.1 of the paper).
//
// Index maps.  A frequency m in [-Lp, Lp] sits at DFT bin k = m mod N; torus rows are
// stored centred (row m + Lp).  Sample theta_t = pi(2t+1)/N, so
//   sum_{m'} X_{m'} e^{i m' theta_t} = sum_k [X_{m'(k)} e^{i pi m'/N}] e^{2 pi i k t / N},
// which is how the phases of eqns dft_phase / idft_spatial enter; phi is the same.
// Phases come from a table ph[k + N - 1] = e^{i pi k / N}, |k| <= N - 1, built in FP64.
#include "ssht_internal.h"

namespace ssht {
namespace {

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

// a * p * scale in the element precision (FP64 arithmetic is avoided on the FP32 path).
template <typename C, typename R>
__device__ __forceinline__ C cmul_d(C a, C p, R scale) {
  C r;
  r.x = (a.x * p.x - a.y * p.y) * scale;
  r.y = (a.x * p.y + a.y * p.x) * scale;
  return r;
}

constexpr int TILE = 32;

// g[b][m+Lp][t] -> h[b][t][k(m)] = g * e^{i pi m / N}, t < L.
template <typename T>
__global__ void inv_theta_to_phi_kernel(int L, const typename Cplx<T>::type* __restrict__ g,
                                        typename Cplx<T>::type* __restrict__ h, const typename Cplx<T>::type* __restrict__ ph) {
  using C = typename Cplx<T>::type;
  __shared__ C tile[TILE][TILE + 1];
  const int Lp = L - 1, N = 2 * L - 1;
  const int b = blockIdx.z;
  const int mi0 = blockIdx.x * TILE, t0 = blockIdx.y * TILE;
  const C* gb = g + (size_t)b * N * N;
  C* hb = h + (size_t)b * L * N;
  for (int r = threadIdx.y; r < TILE; r += blockDim.y) {
    const int mi = mi0 + r, t = t0 + threadIdx.x;
    if (mi < N && t < L) tile[r][threadIdx.x] = gb[(size_t)mi * N + t];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < TILE; r += blockDim.y) {
    const int t = t0 + r, mi = mi0 + threadIdx.x;
    if (mi < N && t < L) {
      const int m = mi - Lp;
      const int k = m >= 0 ? m : m + N;
      hb[(size_t)t * N + k] = cmul_d(tile[threadIdx.x][r], ph[m + N - 1], T(1));
    }
  }
}

// X[b][t][k] (t < L) -> ext[b][m+Lp][t'] for t' < N.
// mode 0 (forward): t' < L: X[t'][k(m)] e^{-i pi m/N}/N, except t' = Lp with odd m+s -> 0;
//                   t' >= L: (-1)^{m+s} X[N-1-t'][k(m)] e^{-i pi m/N}/N.
// mode 1 (adjoint): t' < L: X[t'][k(m)] e^{-i pi m/N}; t' >= L: 0.
template <typename T>
__global__ void fwd_phi_to_theta_kernel(int L, int s, int mode, const typename Cplx<T>::type* __restrict__ X,
                                        typename Cplx<T>::type* __restrict__ ext, const typename Cplx<T>::type* __restrict__ ph) {
  using C = typename Cplx<T>::type;
  __shared__ C tile[TILE][TILE + 1];
  const int Lp = L - 1, N = 2 * L - 1;
  const int b = blockIdx.z;
  const int mi0 = blockIdx.x * TILE, tp0 = blockIdx.y * TILE;
  const C* Xb = X + (size_t)b * L * N;
  C* eb = ext + (size_t)b * N * N;
  // load: rows t' of the output tile map to source rows tsrc; columns are k(m) for the mi tile
  for (int r = threadIdx.y; r < TILE; r += blockDim.y) {
    const int tp = tp0 + r, mi = mi0 + threadIdx.x;
    C v;
    v.x = 0;
    v.y = 0;
    if (tp < N && mi < N) {
      const int m = mi - Lp;
      const int k = m >= 0 ? m : m + N;
      if (tp < L) {
        v = Xb[(size_t)tp * N + k];
      } else if (mode == 0) {
        v = Xb[(size_t)(N - 1 - tp) * N + k];
      }
    }
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  const T inv_n = T(1) / (T)N;
  for (int r = threadIdx.y; r < TILE; r += blockDim.y) {
    const int mi = mi0 + r, tp = tp0 + threadIdx.x;
    if (mi < N && tp < N) {
      const int m = mi - Lp;
      const bool odd = ((m + s) & 1) != 0;
      T scale = (mode == 0) ? inv_n : T(1);
      if (mode == 0 && tp >= L && odd) scale = -scale;
      if (mode == 0 && tp == Lp && odd) scale = T(0);
      eb[(size_t)mi * N + tp] = cmul_d(tile[threadIdx.x][r], ph[-m + N - 1], scale);
    }
  }
}

// Fk[b][mi][k'] -> cx[b][mi][j], j in [0, M): F_{m m''} = Fk[k'(m'')] e^{-i pi m''/N}/N at j = m'' mod M.
template <typename T>
__global__ void fwd_theta_to_conv_kernel(int L, int M, const typename Cplx<T>::type* __restrict__ Fk,
                                         typename Cplx<T>::type* __restrict__ cx, const typename Cplx<T>::type* __restrict__ ph) {
  using C = typename Cplx<T>::type;
  const int Lp = L - 1, N = 2 * L - 1;
  const size_t row = blockIdx.x;  // b * N + mi
  const C* src = Fk + row * N;
  C* dst = cx + row * (size_t)M;
  const T inv_n = T(1) / (T)N;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    int mpp;
    bool have = true;
    if (j <= Lp) mpp = j;
    else if (j >= M - Lp) mpp = j - M;
    else { mpp = 0; have = false; }
    C v;
    v.x = 0;
    v.y = 0;
    if (have) {
      const int k = mpp >= 0 ? mpp : mpp + N;
      v = cmul_d(src[k], ph[-mpp + N - 1], inv_n);
    }
    dst[j] = v;
  }
}

template <typename T>
__global__ void conv_multiply_kernel(int M, size_t rows, typename Cplx<T>::type* __restrict__ cx,
                                     const typename Cplx<T>::type* __restrict__ khat) {
  using C = typename Cplx<T>::type;
  const size_t total = rows * (size_t)M;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const C k = khat[i % M];
    C v = cx[i];
    C r;
    r.x = v.x * k.x - v.y * k.y;
    r.y = v.x * k.y + v.y * k.x;
    cx[i] = r;
  }
}

// y[b][mi][j] -> H[b][mi][m'] = c_{m'} y[m'] / M, c_0 = 2 pi, c_{m'>0} = 4 pi (1/M completes the
// unnormalised inverse FFT of the circular convolution).
template <typename T>
__global__ void conv_to_project_kernel(int L, int M, const typename Cplx<T>::type* __restrict__ y,
                                       typename Cplx<T>::type* __restrict__ H) {
  using C = typename Cplx<T>::type;
  const size_t row = blockIdx.x;
  const T c4 = (T)(4.0 * 3.14159265358979323846 / (double)M);
  for (int mp = threadIdx.x; mp < L; mp += blockDim.x) {
    const T c = (mp == 0) ? T(0.5) * c4 : c4;
    const C v = y[row * (size_t)M + mp];
    C r;
    r.x = c * v.x;
    r.y = c * v.y;
    H[row * (size_t)L + mp] = r;
  }
}

// Adjoint fold: H[b][mi][m'] = H'_{m m'} + (-1)^{m+s} H'_{m,-m'} (m' > 0), H'_{m 0};
// H'_{m m''} = Fk[k'(m'')] e^{-i pi m''/N}.
template <typename T>
__global__ void adj_theta_fold_kernel(int L, int s, const typename Cplx<T>::type* __restrict__ Fk,
                                      typename Cplx<T>::type* __restrict__ H, const typename Cplx<T>::type* __restrict__ ph) {
  using C = typename Cplx<T>::type;
  const int Lp = L - 1, N = 2 * L - 1;
  const size_t row = blockIdx.x;
  const int mi = (int)(row % N);
  const int m = mi - Lp;
  const C* src = Fk + row * N;
  const T sig = ((m + s) & 1) ? T(-1) : T(1);
  for (int mp = threadIdx.x; mp < L; mp += blockDim.x) {
    const C a = cmul_d(src[mp], ph[-mp + N - 1], T(1));
    C r = a;
    if (mp > 0) {
      const C bneg = cmul_d(src[N - mp], ph[mp + N - 1], T(1));
      r.x = a.x + sig * bneg.x;
      r.y = a.y + sig * bneg.y;
    }
    H[row * (size_t)L + mp] = r;
  }
}

// kappa[j] = w_e(p) for the p = j (j <= M/2) or j - M with |p| <= 2 Lp; w_e(p) = 2/(1-p^2), p even.
template <typename T>
__global__ void weight_kernel(int L, int M, typename Cplx<T>::type* __restrict__ kappa) {
  using C = typename Cplx<T>::type;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int p = (j <= M / 2) ? j : j - M;
  double w = 0.0;
  const int ap = p < 0 ? -p : p;
  if (ap <= 2 * (L - 1) && (ap % 2) == 0) w = 2.0 / (1.0 - (double)p * (double)p);
  C v;
  v.x = (T)w;
  v.y = (T)0;
  kappa[j] = v;
}

}  // namespace

template <typename T>
cudaError_t inv_theta_to_phi(const Dims& d, int B, const void* g, void* h, const void* ph, cudaStream_t st) {
  using C = typename Cplx<T>::type;
  dim3 block(TILE, 8), grid((d.N + TILE - 1) / TILE, (d.L + TILE - 1) / TILE, B);
  inv_theta_to_phi_kernel<T><<<grid, block, 0, st>>>(d.L, (const C*)g, (C*)h, (const C*)ph);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fwd_phi_to_theta(const Dims& d, int s, int B, int mode, const void* X, void* ext, const void* ph,
                             cudaStream_t st) {
  using C = typename Cplx<T>::type;
  dim3 block(TILE, 8), grid((d.N + TILE - 1) / TILE, (d.N + TILE - 1) / TILE, B);
  fwd_phi_to_theta_kernel<T><<<grid, block, 0, st>>>(d.L, s, mode, (const C*)X, (C*)ext, (const C*)ph);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fwd_theta_to_conv(const Dims& d, int B, const void* Fk, void* cx, const void* ph, cudaStream_t st) {
  using C = typename Cplx<T>::type;
  const int threads = 256;
  const unsigned grid = (unsigned)((size_t)B * d.N);
  fwd_theta_to_conv_kernel<T><<<grid, threads, 0, st>>>(d.L, d.M, (const C*)Fk, (C*)cx, (const C*)ph);
  return cudaGetLastError();
}

template <typename T>
cudaError_t conv_multiply(const Dims& d, int B, void* cx, const void* khat, cudaStream_t st) {
  using C = typename Cplx<T>::type;
  const size_t rows = (size_t)B * d.N;
  const size_t total = rows * d.M;
  const int threads = 256;
  const unsigned blocks = (unsigned)std::min<size_t>((total + threads - 1) / threads, 152 * 64);
  conv_multiply_kernel<T><<<blocks, threads, 0, st>>>(d.M, rows, (C*)cx, (const C*)khat);
  return cudaGetLastError();
}

template <typename T>
cudaError_t conv_to_project(const Dims& d, int B, const void* y, void* H, cudaStream_t st) {
  using C = typename Cplx<T>::type;
  const int threads = 128;
  const unsigned grid = (unsigned)((size_t)B * d.N);
  conv_to_project_kernel<T><<<grid, threads, 0, st>>>(d.L, d.M, (const C*)y, (C*)H);
  return cudaGetLastError();
}

template <typename T>
cudaError_t adj_theta_fold(const Dims& d, int s, int B, const void* Fk, void* H, const void* ph, cudaStream_t st) {
  using C = typename Cplx<T>::type;
  const int threads = 128;
  const unsigned grid = (unsigned)((size_t)B * d.N);
  adj_theta_fold_kernel<T><<<grid, threads, 0, st>>>(d.L, s, (const C*)Fk, (C*)H, (const C*)ph);
  return cudaGetLastError();
}

template <typename T>
cudaError_t make_weight_kernel(const Dims& d, void* kappa, cudaStream_t st) {
  using C = typename Cplx<T>::type;
  const int threads = 256;
  weight_kernel<T><<<(d.M + threads - 1) / threads, threads, 0, st>>>(d.L, d.M, (C*)kappa);
  return cudaGetLastError();
}

#define SSHT_INST(T)                                                                                        \
  template cudaError_t inv_theta_to_phi<T>(const Dims&, int, const void*, void*, const void*, cudaStream_t); \
  template cudaError_t fwd_phi_to_theta<T>(const Dims&, int, int, int, const void*, void*, const void*,     \
                                           cudaStream_t);                                                   \
  template cudaError_t fwd_theta_to_conv<T>(const Dims&, int, const void*, void*, const void*, cudaStream_t); \
  template cudaError_t conv_multiply<T>(const Dims&, int, void*, const void*, cudaStream_t);                \
  template cudaError_t conv_to_project<T>(const Dims&, int, const void*, void*, cudaStream_t);              \
  template cudaError_t adj_theta_fold<T>(const Dims&, int, int, const void*, void*, const void*, cudaStream_t); \
  template cudaError_t make_weight_kernel<T>(const Dims&, void*, cudaStream_t);
SSHT_INST(double)
SSHT_INST(float)
#undef SSHT_INST

}  // namespace ssht
