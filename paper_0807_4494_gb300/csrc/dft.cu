// Batched discrete Fourier transforms of odd length N = 2L-1 (the torus sampling of eqns
// nodes_theta / nodes_phi, Sec. 3.4.1) in FP32, by Bluestein's chirp-z algorithm with a
// power-of-two FFT in shared memory.
//
//   X_k = sum_{n<N} x_n e^{-+ 2 pi i n k / N}
//       = c_k sum_n (x_n c_n) conj(c)_{k-n},   c_j = e^{-+ i pi j^2 / N}   (nk = (n^2+k^2-(k-n)^2)/2)
//
// The sum over n is a linear convolution of length 2N-1, done as a circular convolution of
// length M = 2^p >= 2N-1: one forward FFT of the chirped row, a pointwise product with the
// precomputed spectrum of the chirp kernel (1/M folded in), one inverse FFT.  The FFTs are
// Stockham autosort passes of radix 16 (last pass radix 2/4/8 when M is not a power of 16),
// one pass per shared-memory round trip, each thread holding one radix-R butterfly in registers.
// Chirps, kernel spectra and twiddles are computed in FP64 on the host and stored in FP32.
// Rows of length N <= 32 use a direct O(N^2) sum instead.
//
// This replaces cuFFT for the odd lengths, which cuFFT handles with slow prime-factor kernels
// (2047 = 23 x 89: 9x slower than length 2048 on this GPU).
#include "ssht_internal.h"

#include <cmath>
#include <complex>
#include <vector>

namespace ssht {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward, sign -1) or +i (inverse, sign +1)
template <int SIGN>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int SIGN>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// In-place DFT4 of (a0, a1, a2, a3), natural order out.
template <int SIGN>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi<SIGN>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

__device__ __forceinline__ float2 tw16(int k, int sign) {
  // e^{sign 2 pi i k / 16}, k in [0, 16)
  const float c[16] = {1.f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f, 0.f,
                       -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f, -1.f,
                       -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f, 0.f,
                       0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
  const float s = c[(k + 12) & 15];  // sin(2 pi k/16) = cos(2 pi (k-4)/16)
  return make_float2(c[k & 15], sign < 0 ? -s : s);
}

// In-register DFT of size R (2, 4, 8, 16), input v[n], output v[k] in natural order.
template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2* v) {
  if (R == 2) {
    dft2<SIGN>(v[0], v[1]);
  } else if (R == 4) {
    dft4<SIGN>(v[0], v[1], v[2], v[3]);
  } else if (R == 8) {
    // n = 2 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W8^{n2 k1}, DFT2 over n2
    float2 a[4] = {v[0], v[2], v[4], v[6]}, b[4] = {v[1], v[3], v[5], v[7]};
    dft4<SIGN>(a[0], a[1], a[2], a[3]);
    dft4<SIGN>(b[0], b[1], b[2], b[3]);
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) b[k1] = cmul(b[k1], tw16(2 * k1, SIGN));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      v[k1] = cadd(a[k1], b[k1]);
      v[k1 + 4] = csub(a[k1], b[k1]);
    }
  } else {
    // n = 4 n1 + n2, k = k1 + 4 k2
    float2 y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      y[n2][0] = v[n2];
      y[n2][1] = v[4 + n2];
      y[n2][2] = v[8 + n2];
      y[n2][3] = v[12 + n2];
      dft4<SIGN>(y[n2][0], y[n2][1], y[n2][2], y[n2][3]);
    }
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) y[n2][k1] = cmul(y[n2][k1], tw16(n2 * k1, SIGN));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 a0 = y[0][k1], a1 = y[1][k1], a2 = y[2][k1], a3 = y[3][k1];
      dft4<SIGN>(a0, a1, a2, a3);
      v[k1] = a0;
      v[k1 + 4] = a1;
      v[k1 + 8] = a2;
      v[k1 + 12] = a3;
    }
  }
}

// Shared-memory index with one pad word per 16 complex values (spreads the strided accesses of
// the Stockham passes over the banks).
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// One Stockham pass of radix R over a row of M values in shared memory, T threads per row.
template <int M, int R, int SIGN, int T>
__device__ __forceinline__ void stockham_pass(float2* buf, int Ns, int tid, const float2* __restrict__ tw) {
  constexpr int J = M / R;           // butterflies
  constexpr int PER = (J + T - 1) / T;
  float2 v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid + q * T;
    if (j < J) {
      const int jm = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 x = buf[pidx(j + r * J)];
        if (r > 0 && Ns > 1) {
          float2 w = __ldg(&tw[jm * r * (M / (Ns * R))]);  // e^{-2 pi i jm r / (Ns R)}
          if (SIGN > 0) w = conjf2(w);
          x = cmul(x, w);
        }
        v[q][r] = x;
      }
      dft_reg<R, SIGN>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid + q * T;
    if (j < J) {
      const int jm = j % Ns;
      const int d = (j / Ns) * Ns * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pidx(d + r * Ns)] = v[q][r];
    }
  }
  __syncthreads();
}

// Full FFT of size M (natural order in and out) by T = M/16 threads (M >= 128).
template <int M, int SIGN>
__device__ __forceinline__ void fft_smem(float2* buf, int tid, const float2* __restrict__ tw) {
  constexpr int T = M / 16;
  int Ns = 1;
  int rem = M;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    if (rem >= 16) {
      stockham_pass<M, 16, SIGN, T>(buf, Ns, tid, tw);
      Ns *= 16;
      rem /= 16;
    }
  }
  if (rem == 8) stockham_pass<M, 8, SIGN, T>(buf, Ns, tid, tw);
  else if (rem == 4) stockham_pass<M, 4, SIGN, T>(buf, Ns, tid, tw);
  else if (rem == 2) stockham_pass<M, 2, SIGN, T>(buf, Ns, tid, tw);
}

struct BluesteinTables {
  const float2* chirp;   // c_n = e^{-i pi n^2 / N}, n < N
  const float2* khat_f;  // FFT_M(conj chirp kernel)/M for the forward DFT (sign -1)
  const float2* khat_i;  // the same for the inverse DFT (sign +1)
  const float2* tw;      // e^{-2 pi i k / M}, k < M
};

// Rows of length N: out[row][k] = sum_n in[row][n] e^{SIGN 2 pi i n k / N}.  G rows per CTA, each
// by M/16 threads.  in and out may be the same buffer.
template <int M, int SIGN>
__global__ void __launch_bounds__(M >= 8192 ? 512 : 256) bluestein_kernel(int N, long long nrows, const float2* in, float2* out,
                                                       BluesteinTables tb) {
  constexpr int T = M / 16;
  constexpr int G = (256 / T) > 0 ? 256 / T : 1;
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / T, tid = threadIdx.x % T;
  float2* buf = sm + g * (M + M / 16);
  const float2* khat = SIGN < 0 ? tb.khat_f : tb.khat_i;
  for (long long row0 = (long long)blockIdx.x * G; row0 < nrows; row0 += (long long)gridDim.x * G) {
    const long long row = row0 + g;
    const bool active = row < nrows;
    const float2* x = in + (size_t)(active ? row : 0) * N;
    // 1. chirp the row and zero-pad to M
    for (int n = tid; n < M; n += T) {
      float2 v = make_float2(0.f, 0.f);
      if (active && n < N) {
        float2 c = __ldg(&tb.chirp[n]);
        if (SIGN > 0) c = conjf2(c);
        v = cmul(x[n], c);
      }
      buf[pidx(n)] = v;
    }
    __syncthreads();
    // 2. forward FFT, 3. product with the kernel spectrum, 4. inverse FFT
    fft_smem<M, -1>(buf, tid, tb.tw);
    for (int k = tid; k < M; k += T) buf[pidx(k)] = cmul(buf[pidx(k)], __ldg(&khat[k]));
    __syncthreads();
    fft_smem<M, 1>(buf, tid, tb.tw);
    // 5. chirp the result
    if (active) {
      float2* y = out + (size_t)row * N;
      for (int k = tid; k < N; k += T) {
        float2 c = __ldg(&tb.chirp[k]);
        if (SIGN > 0) c = conjf2(c);
        y[k] = cmul(buf[pidx(k)], c);
      }
    }
    __syncthreads();
  }
}

// Direct DFT for short rows (N <= 32): one warp per row, twiddles e^{-2 pi i k / N} from a table.
template <int SIGN>
__global__ void direct_dft_kernel(int N, long long nrows, const float2* in, float2* out, const float2* __restrict__ twN) {
  __shared__ float2 xs[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long row = (long long)blockIdx.x * 8 + w; row < nrows; row += (long long)gridDim.x * 8) {
    xs[w][lane] = lane < N ? in[(size_t)row * N + lane] : make_float2(0.f, 0.f);
    __syncwarp();
    if (lane < N) {
      float2 acc = make_float2(0.f, 0.f);
      for (int n = 0; n < N; ++n) {
        float2 t = twN[(lane * n) % N];
        if (SIGN > 0) t = conjf2(t);
        acc = cadd(acc, cmul(xs[w][n], t));
      }
      out[(size_t)row * N + lane] = acc;
    }
    __syncwarp();
  }
}

// Host FFT in FP64 (iterative radix-2), used only to build the kernel spectra.
void host_fft(std::vector<std::complex<double>>& a, int sign) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  const double pi = 3.14159265358979323846;
  for (size_t len = 2; len <= n; len <<= 1) {
    const double ang = sign * 2 * pi / (double)len;
    for (size_t i = 0; i < n; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
        const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

}  // namespace

struct DftPlan {
  int N = 0, M = 0;
  float2* chirp = nullptr;
  float2* khat_f = nullptr;
  float2* khat_i = nullptr;
  float2* tw = nullptr;
  float2* twN = nullptr;  // direct DFT twiddles (N <= 32)
  size_t bytes = 0;
};

cudaError_t dft_setup(DftPlan** out, int N) {
  *out = nullptr;
  DftPlan* p = new DftPlan();
  p->N = N;
  const double pi = 3.14159265358979323846;
  cudaError_t e = cudaSuccess;
  if (N <= 32) {
    std::vector<float2> t(N);
    for (int k = 0; k < N; ++k) t[k] = make_float2((float)std::cos(-2 * pi * k / N), (float)std::sin(-2 * pi * k / N));
    if ((e = cudaMalloc(&p->twN, N * sizeof(float2))) != cudaSuccess) goto fail;
    if ((e = cudaMemcpy(p->twN, t.data(), N * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess) goto fail;
    p->bytes = N * sizeof(float2);
    *out = p;
    return cudaSuccess;
  }
  {
    int M = 128;
    while (M < 2 * N - 1) M <<= 1;
    p->M = M;
    std::vector<float2> chirp(N), tw(M), kf(M), ki(M);
    for (int n = 0; n < N; ++n) {
      const long long r = ((long long)n * n) % (2LL * N);  // e^{-i pi n^2/N} depends on n^2 mod 2N
      const double a = -pi * (double)r / (double)N;
      chirp[n] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (int k = 0; k < M; ++k)
      tw[k] = make_float2((float)std::cos(-2 * pi * k / M), (float)std::sin(-2 * pi * k / M));
    // kernel b_j = conj(c_j) at j mod M, |j| < N; spectrum / M.  Forward DFT uses b, inverse conj(b).
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<std::complex<double>> b(M, 0.0);
      for (int j = -(N - 1); j <= N - 1; ++j) {
        const long long jj = (long long)j * j % (2LL * N);
        const double a = (dir == 0 ? 1.0 : -1.0) * pi * (double)jj / (double)N;
        b[(j + M) % M] = std::complex<double>(std::cos(a), std::sin(a));
      }
      host_fft(b, -1);
      std::vector<float2>& dst = dir == 0 ? kf : ki;
      for (int k = 0; k < M; ++k) dst[k] = make_float2((float)(b[k].real() / M), (float)(b[k].imag() / M));
    }
    float2** bufs[] = {&p->chirp, &p->tw, &p->khat_f, &p->khat_i};
    const std::vector<float2>* src[] = {&chirp, &tw, &kf, &ki};
    for (int i = 0; i < 4; ++i) {
      const size_t bytes = src[i]->size() * sizeof(float2);
      if ((e = cudaMalloc(bufs[i], bytes)) != cudaSuccess) goto fail;
      if ((e = cudaMemcpy(*bufs[i], src[i]->data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess) goto fail;
      p->bytes += bytes;
    }
    const int smem_rows = (M / 16 >= 256) ? 1 : 256 / (M / 16);
    const int smem = smem_rows * (M + M / 16) * (int)sizeof(float2);
#define SSHT_DFT_ATTR(MM)                                                                                    \
  if (M == MM) {                                                                                             \
    if ((e = cudaFuncSetAttribute(bluestein_kernel<MM, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != \
        cudaSuccess) goto fail;                                                                              \
    if ((e = cudaFuncSetAttribute(bluestein_kernel<MM, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=  \
        cudaSuccess) goto fail;                                                                              \
  }
    SSHT_DFT_ATTR(128) SSHT_DFT_ATTR(256) SSHT_DFT_ATTR(512) SSHT_DFT_ATTR(1024) SSHT_DFT_ATTR(2048)
    SSHT_DFT_ATTR(4096) SSHT_DFT_ATTR(8192)
#undef SSHT_DFT_ATTR
  }
  *out = p;
  return cudaSuccess;
fail:
  dft_destroy(p);
  return e;
}

void dft_destroy(DftPlan* p) {
  if (!p) return;
  void* q[] = {p->chirp, p->khat_f, p->khat_i, p->tw, p->twN};
  for (void* x : q)
    if (x) cudaFree(x);
  delete p;
}

size_t dft_bytes(const DftPlan* p) { return p ? p->bytes : 0; }

cudaError_t dft_rows(const DftPlan* p, int sign, long long nrows, const void* in, void* out, cudaStream_t st) {
  if (nrows <= 0) return cudaSuccess;
  const int N = p->N;
  if (N <= 32) {
    const long long blocks = std::min<long long>((nrows + 7) / 8, 152LL * 64);
    if (sign < 0)
      direct_dft_kernel<-1><<<(unsigned)blocks, 256, 0, st>>>(N, nrows, (const float2*)in, (float2*)out, p->twN);
    else
      direct_dft_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(N, nrows, (const float2*)in, (float2*)out, p->twN);
    return cudaGetLastError();
  }
  BluesteinTables tb{p->chirp, p->khat_f, p->khat_i, p->tw};
  const int M = p->M;
  const int T = M / 16, G = (T >= 256) ? 1 : 256 / T;
  const int threads = T * G;
  const int smem = G * (M + M / 16) * (int)sizeof(float2);
  const long long blocks = std::min<long long>((nrows + G - 1) / G, 152LL * 32);
#define SSHT_DFT_LAUNCH(MM)                                                                                   \
  if (M == MM) {                                                                                              \
    if (sign < 0)                                                                                             \
      bluestein_kernel<MM, -1><<<(unsigned)blocks, threads, smem, st>>>(N, nrows, (const float2*)in, (float2*)out, tb); \
    else                                                                                                      \
      bluestein_kernel<MM, 1><<<(unsigned)blocks, threads, smem, st>>>(N, nrows, (const float2*)in, (float2*)out, tb);  \
    return cudaGetLastError();                                                                                \
  }
  SSHT_DFT_LAUNCH(128) SSHT_DFT_LAUNCH(256) SSHT_DFT_LAUNCH(512) SSHT_DFT_LAUNCH(1024) SSHT_DFT_LAUNCH(2048)
  SSHT_DFT_LAUNCH(4096) SSHT_DFT_LAUNCH(8192)
#undef SSHT_DFT_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace ssht
