// Fused torus passes of the FP32 / tensor-core plans: the odd-length DFTs along theta and phi
// (eqns dft_spatial / idft_spatial, Sec. 3.4.1) with the extension, phase, weight convolution and
// transposition steps folded into their loads and stores.
//
// DFT core.  A row of length N = 2L-1 is transformed by Bluestein's algorithm: the
// chirped row goes through a forward FFT of size M = 2^p >= 2N-1, a product with the chirp
// kernel's spectrum and an inverse FFT.  The FFTs are Stockham autosort passes (radix 16, last
// pass radix 2/4/8) executed by T = M/16 threads per row; the first pass reads its inputs through a
// source functor and the last pass hands its outputs to a sink functor, so the chirp and kernel
// products and the kernels' own input/output transforms cost no extra shared-memory round trip.
// Twiddles are staged in shared memory once per CTA, one table per pass laid out so that a warp
// reads consecutive words.
//
// Pairing.  Along theta every phi-frequency column m is even or odd about theta = 0 (parity
// (-1)^{m+s}, Sec. 3.2) and adjacent columns have opposite parities, so one complex DFT serves
// two columns: z = x_m + x_{m+1} is transformed and the halves are separated afterwards,
//   x_m(theta_t) = (z(theta_t) + s_m z(theta_{N-1-t}))/2,  x_{m+1}(theta_t) = (z(theta_t) - s_m z(theta_{N-1-t}))/2,
// (theta_{N-1-t} = 2 pi - theta_t) and in the frequency domain likewise with k -> -k.
//
// Kernels (b = field, rows of the torus stored centred, m + Lp):
//   inverse_theta:  F[b][m][m'] (m' in [0,L), eqn fourier_coeff) -> h[b][t][m mod N] (t < L),
//                   i.e. theta synthesis with the extension eqn Ffourier_sym and both phases of
//                   eqn idft_spatial; one pair of columns per row group.
//   rows (phi):     h[b][t][:] -> f[b][t][:] (inverse), f[b][t][:] -> X (forward/adjoint), stored
//                   by pairs of columns: X[b][p][t][j], column m + Lp = 2p + j (N + 1 rows a field,
//                   the last pair half used), so that a store carries two columns of one ring and
//                   the theta passes read a pair with one 16-byte load.
//   forward_theta:  X (a pair of columns) -> H[b][m][m'] (m' in [0,L)): per-m parity extension,
//                   theta DFT, then the sin(theta) weight convolution as a zero-padded circular
//                   convolution of length M in the same shared-memory buffer, and the fold of
//                   m' < 0.  Tensor-core plans: the projection's split data tiles in place of H
//                   (put_tile), so that the forward transform needs no separate data packing.
//   adjoint_theta:  X (one column) -> H[b][m][m'] or the data tiles: theta DFT of the unextended
//                   rings, fold of m' < 0.
#include "ssht_internal.h"
#include "bounds.cuh"
#include "tc_common.cuh"

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
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
template <int SIGN>
__device__ __forceinline__ float2 mul_mi(float2 a) {  // * e^{SIGN i pi/2}
  return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi<SIGN>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// e^{SIGN 2 pi i k/16}, k a compile-time constant after unrolling
template <int SIGN>
__device__ __forceinline__ float2 w16(int k) {
  const float c0 = 1.f, c1 = 0.92387953251128674f, c2 = 0.70710678118654752f, c3 = 0.38268343236508977f;
  const int kk = k & 15;
  const float cs[16] = {c0, c1, c2, c3, 0.f, -c3, -c2, -c1, -c0, -c1, -c2, -c3, 0.f, c3, c2, c1};
  const float s = cs[(kk + 12) & 15];
  return make_float2(cs[kk], SIGN < 0 ? -s : s);
}

// R-point DFT on registers.  Z (R = 16 only): 1 when inputs 8..15 are zero (the zero-padded half
// of a Bluestein row), 2 when only outputs 0..7 are wanted (the half of the spectrum a Bluestein
// row keeps); the work that only touches the absent half is left out.
template <int R, int SIGN, int Z = 0>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (R == 2) {
    const float2 t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  } else if constexpr (R == 4) {
    dft4<SIGN>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    float2 a0 = v[0], a1 = v[2], a2 = v[4], a3 = v[6], b0 = v[1], b1 = v[3], b2 = v[5], b3 = v[7];
    dft4<SIGN>(a0, a1, a2, a3);
    dft4<SIGN>(b0, b1, b2, b3);
    b1 = cmul(b1, w16<SIGN>(2));
    b2 = mul_mi<SIGN>(b2);  // w16(4)
    b3 = cmul(b3, w16<SIGN>(6));
    v[0] = cadd(a0, b0); v[4] = csub(a0, b0);
    v[1] = cadd(a1, b1); v[5] = csub(a1, b1);
    v[2] = cadd(a2, b2); v[6] = csub(a2, b2);
    v[3] = cadd(a3, b3); v[7] = csub(a3, b3);
  } else {
    // 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      if constexpr (Z == 1) {
        // inputs n1 = 2, 3 are zero
        const float2 a0 = v[n2], a1 = v[4 + n2], ia1 = mul_mi<SIGN>(a1);
        v[n2] = cadd(a0, a1);
        v[4 + n2] = cadd(a0, ia1);
        v[8 + n2] = csub(a0, a1);
        v[12 + n2] = csub(a0, ia1);
      } else {
        dft4<SIGN>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
      }
    }
    // now v[4 k1 + n2] holds Y[n2][k1]
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) {
        if (n2 * k1 == 4) v[4 * k1 + n2] = mul_mi<SIGN>(v[4 * k1 + n2]);
        else v[4 * k1 + n2] = cmul(v[4 * k1 + n2], w16<SIGN>(n2 * k1));
      }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      if constexpr (Z == 2) {
        // outputs k2 = 0, 1 only
        float2& a0 = v[4 * k1 + 0];
        float2& a1 = v[4 * k1 + 1];
        const float2 a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
        const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi<SIGN>(csub(a1, a3));
        a0 = cadd(t0, t2);
        a1 = cadd(t1, t3);
      } else {
        dft4<SIGN>(v[4 * k1 + 0], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
      }
    }
    // v[4 k1 + k2] holds X[k1 + 4 k2]: transpose the 4x4 block into natural order
    float2 t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = t[i];
  }
}

__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// Pass structure of an FFT of size M: P16 radix-16 passes, then one pass of radix REST (1 = none).
// Pass i has stride NS = 16^i.  Twiddles of pass i >= 1 sit in a table of (R - 1) * NS entries,
// entry (r - 1) * NS + j' = e^{-2 pi i j' r / (NS R)}, so that consecutive threads read
// consecutive words; the tables of all passes are stored back to back (about M entries).
__host__ __device__ constexpr int pow16(int i) { return i == 0 ? 1 : 16 * pow16(i - 1); }
template <int M> struct Plan16 {
  static constexpr int P16 = (M >= 4096) ? 3 : (M >= 256) ? 2 : 1;
  static constexpr int REST = M >> (4 * P16);
  static constexpr int NP = P16 + (REST > 1 ? 1 : 0);
  __host__ __device__ static constexpr int radix(int i) { return i < P16 ? 16 : REST; }
  __host__ __device__ static constexpr int off(int i) { return i <= 1 ? 0 : off(i - 1) + (radix(i - 1) - 1) * pow16(i - 1); }
  static constexpr int TW = off(NP);  // table entries
};

// One Stockham pass of radix R and stride NS: inputs through src(i) (first pass) or shared memory,
// outputs through sink(k, v) (last pass) or shared memory.  twp: this pass's twiddle table.
// Z = 1 (first pass, read from src): inputs at positions >= M/2 (r >= R/2) are zero and not read;
// Z = 2 (last pass, written to sink): outputs at positions >= M/2 are not wanted.
template <int M, int R, int NS, int SIGN, bool FROM_SRC, bool TO_SINK, int Z, class Src, class Sink>
__device__ __forceinline__ void pass(float2* buf, int tid, const float2* twp, Src& src, Sink& sink) {
  constexpr int T = M / 16;
  constexpr int J = M / R;
  constexpr int PER = J / T;
  constexpr bool ZIN = FROM_SRC && Z == 1, ZOUT = TO_SINK && Z == 2;
  float2 v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid + q * T;
    const int jm = j & (NS - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 x;
      if constexpr (ZIN) {
        if (r >= R / 2) {
          v[q][r] = make_float2(0.f, 0.f);
          continue;
        }
      }
      if constexpr (FROM_SRC) x = src(j + r * J);
      else x = buf[pidx(j + r * J)];
      if constexpr (NS > 1) {
        if (r > 0) {
          float2 w = twp[(r - 1) * NS + jm];
          if (SIGN > 0) w = conjf2(w);
          x = cmul(x, w);
        }
      }
      v[q][r] = x;
    }
    dft_reg<R, SIGN, ZIN ? 1 : ZOUT ? 2 : 0>(v[q]);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid + q * T;
    const int d = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (ZOUT) {
        if (r >= R / 2) continue;
      }
      if constexpr (TO_SINK) sink(d + r * NS, v[q][r]);
      else buf[pidx(d + r * NS)] = v[q][r];
    }
  }
  __syncthreads();
}

// Passes [I, IEND) of an FFT of size M and sign SIGN; pass 0 reads src, pass NP - 1 writes sink.
// Z: 1 when the inputs at positions >= M/2 are zero, 2 when only outputs below M/2 are wanted.
template <int M, int SIGN, int I, int IEND, int Z = 0, class Src, class Sink>
__device__ __forceinline__ void run_range(float2* buf, int tid, const float2* tw, Src& src, Sink& sink) {
  if constexpr (I < IEND) {
    using P = Plan16<M>;
    pass<M, P::radix(I), pow16(I), SIGN, I == 0, I == P::NP - 1, Z>(buf, tid, tw + P::off(I), src, sink);
    run_range<M, SIGN, I + 1, IEND, Z>(buf, tid, tw, src, sink);
  }
}

// FFT of size M (sign SIGN, unnormalised): inputs through src(i), outputs through sink(k, v),
// both in natural order.  Ends with a barrier; buf is free afterwards.
template <int M, int SIGN, class Src, class Sink>
__device__ __forceinline__ void fft(float2* buf, int tid, const float2* tw, Src src, Sink sink) {
  run_range<M, SIGN, 0, Plan16<M>::NP>(buf, tid, tw, src, sink);
}

// The last pass of an FFT of sign SA fused with the first pass of the next FFT, of sign SB, with a
// pointwise map op(k, v) on the spectrum in between.  In both passes thread tid owns the positions
// tid + T c, c < 16 (the last pass writes j + r NS with j < NS, NS a multiple of T; the first pass
// reads tid + r T), so the map runs on registers and the spectrum never goes to shared memory.
template <int M, int SA, int SB, class Op>
__device__ __forceinline__ void boundary(float2* buf, int tid, const float2* tw, Op& op) {
  using P = Plan16<M>;
  constexpr int I = P::NP - 1, R = P::radix(I), NS = pow16(I), T = M / 16, J = M / R, PER = J / T;
  static_assert(I >= 1 && NS % T == 0 && PER * R == 16, "pass geometry");
  const float2* twp = tw + P::off(I);
  float2 v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = tid + q * T;
    const int jm = j & (NS - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 x = buf[pidx(j + r * J)];
      if (r > 0) {
        float2 w = twp[(r - 1) * NS + jm];
        if (SA > 0) w = conjf2(w);
        x = cmul(x, w);
      }
      v[q][r] = x;
    }
    dft_reg<R, SA>(v[q]);
  }
  float2 u[16];
#pragma unroll
  for (int q = 0; q < PER; ++q)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      constexpr int S = NS / T;
      const int c = q + r * S;
      u[c] = op(tid + T * c, v[q][r]);
    }
  dft_reg<16, SB>(u);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[pidx(16 * tid + r)] = u[r];
  __syncthreads();
}

struct NoSrc {
  __device__ float2 operator()(int) const { return make_float2(0.f, 0.f); }
};
struct NoSink {
  __device__ void operator()(int, float2) const {}
};

struct TorusTables {
  const float2* chirp;  // e^{-i pi n^2/N}, n < N
  const float2* khat_f; // spectrum of the forward-DFT chirp kernel, / M
  const float2* khat_i; // the same for the inverse DFT
  const float2* tw;     // per-pass twiddle tables (Plan16<M>::TW entries)
  const float2* what;   // spectrum of the even sin(theta) weight w_e (zero-padded, length M), / M
  const float2* ph;     // e^{i pi k/N}, |k| < N, at k + N - 1
  const float2* chirp_ph;  // chirp[k] e^{-i pi m/N}, m = k (k < L) or k - N: the forward DFT's
                           // output chirp with the phase of eqn dft_spatial, one rounding
  const float2* khat_c;    // spectrum of the forward-DFT chirp kernel for centred outputs, / M
  const float2* chirp_c;   // at k = m mod M, |m| < L: e^{-i pi (m^2 + m)/N} / N; 0 for L <= k <= M - L
};

// Extents of a pass's input and output buffers in float2 elements (the index checks of builds with
// SSHT_DEBUG).
struct Ext {
  long long in, out;
};

// Bluestein DFT of one row: out_k = sum_n in_n e^{SIGN 2 pi i n k/N}.  in through src(n) (n < N),
// out through sink(k, v) (k < N).  buf: M (+pad) values; ends with buf free.  PHASE (forward DFTs
// only): out_k also carries e^{-i pi m/N}, m = k or k - N.  IN_PHASE (inverse DFTs only): in_n
// is src(n) e^{i pi m/N}, m = n or n - N (one table, the conjugate of the forward's combined
// output chirp).  The chirped row's FFT and the inverse FFT of its product with the kernel's
// spectrum meet in one fused pass.
template <int M, int SIGN, bool PHASE = false, bool IN_PHASE = false, class Src, class Sink>
__device__ __forceinline__ void bluestein(float2* buf, int tid, const float2* tw, const TorusTables& tb, int N, Src src,
                                          Sink sink) {
  static_assert(!PHASE || SIGN < 0, "the combined output table is the forward chirp's");
  static_assert(!IN_PHASE || SIGN > 0, "the combined input table is the inverse chirp's");
  const float2* khat = SIGN < 0 ? tb.khat_f : tb.khat_i;
  auto in = [&](int n) {
    if (n >= N) return make_float2(0.f, 0.f);
    float2 c = __ldg(IN_PHASE ? &tb.chirp_ph[n] : &tb.chirp[n]);
    if (SIGN > 0) c = conjf2(c);
    return cmul(src(n), c);
  };
  auto mid = [&](int k, float2 v) { return cmul(v, __ldg(&khat[k])); };
  auto out = [&](int k, float2 v) {
    if (k < N) {
      float2 c = __ldg(PHASE ? &tb.chirp_ph[k] : &tb.chirp[k]);
      if (SIGN > 0) c = conjf2(c);
      sink(k, cmul(v, c));
    }
  };
  NoSrc none_in;
  NoSink none_out;
  // the chirped row is zero from N <= M/2 on, and only outputs below N are kept
  constexpr int NP = Plan16<M>::NP;
  run_range<M, -1, 0, NP - 1, 1>(buf, tid, tw, in, none_out);
  boundary<M, -1, 1>(buf, tid, tw, mid);
  run_range<M, 1, 1, NP, 2>(buf, tid, tw, none_in, out);
}

// Ask L2 for [p, p + bytes), one 128-byte line a thread of the row group (T threads): the input of
// the row group's next row, fetched while the current row is transformed.  Every line named holds
// bytes of the buffer.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes, int tid, int T) {
  const unsigned long long a = (unsigned long long)p, first = a >> 7, last = (a + bytes - 1) >> 7;
  for (unsigned long long l = first + tid; l <= last; l += T) asm volatile("prefetch.L2 [%0];" ::"l"(l << 7));
}

#ifndef SSHT_TORUS_MINB
#define SSHT_TORUS_MINB 3  // resident CTAs of 256 threads an SM the passes' registers are sized for
#endif

template <int M> struct Geo {
  static constexpr int T = M / 16;
  static constexpr int G = (T >= 256) ? 1 : 256 / T;  // row groups per CTA
  static constexpr int THREADS = T * G;
  static constexpr int BUF = M + M / 16;
  static constexpr int MINB = THREADS >= 512 ? 1 : SSHT_TORUS_MINB;  // CTAs per SM the register budget is sized for
  static constexpr int SMEM = (Plan16<M>::TW + G * BUF) * 8;
};

// Stage the twiddle table in shared memory; returns the row group's buffer.
template <int M>
__device__ __forceinline__ float2* setup_smem(const TorusTables& tb, float2** tw_out) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  for (int k = threadIdx.x; k < Plan16<M>::TW; k += blockDim.x) tw[k] = __ldg(&tb.tw[k]);
  __syncthreads();
  *tw_out = tw;
  return sm + Plan16<M>::TW + (threadIdx.x / Geo<M>::T) * Geo<M>::BUF;
}

// ---------------------------------------------------------------------------------------------
// inverse theta synthesis: F half rows -> h (phi-DFT input), one pair of columns per row group
// ---------------------------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(Geo<M>::THREADS, Geo<M>::MINB) inverse_theta_kernel(int L, int s, int B, const float2* __restrict__ F,
                                                                       float2* __restrict__ h, TorusTables tb, Ext ext) {
  float2* tw;
  float2* buf = setup_smem<M>(tb, &tw);
  const int Lp = L - 1, N = 2 * L - 1;
  const int tid = threadIdx.x % Geo<M>::T;
  const long long npairs = (long long)B * L;  // pair p: m = -Lp + 2p (and m + 1 when p < Lp)
  for (long long u0 = (long long)blockIdx.x * Geo<M>::G; u0 < npairs; u0 += (long long)gridDim.x * Geo<M>::G) {
    const long long u = u0 + threadIdx.x / Geo<M>::T;
    const bool active = u < npairs;
    const int b = active ? (int)(u / L) : 0, p = active ? (int)(u % L) : 0;
    const int m = -Lp + 2 * p;
    const bool two = p < Lp;
    const float sig = ((m + s) & 1) ? -1.f : 1.f;  // parity of column m; column m+1 has -sig
    const float2* F0 = F + ((size_t)b * N + (m + Lp)) * L;
    const float2* F1 = F0 + L;
    {
      const long long un = u + (long long)gridDim.x * Geo<M>::G;
      if (un < npairs) {
        const int bn = (int)(un / L), pn = (int)(un % L);
        prefetch_l2(F + ((size_t)bn * N + 2 * pn) * L, (pn < Lp ? 2 : 1) * (size_t)L * sizeof(float2), tid, Geo<M>::T);
      }
    }
    auto src = [&](int n) {
      if (!active) return make_float2(0.f, 0.f);
      const int mp = n < L ? n : N - n;  // theta frequency m' (>= 0) of DFT bin n
      const long long i0 = (F0 - F) + mp;
      float2 a = in_bounds(i0, ext.in, kbInverseThetaIn) ? F0[mp] : make_float2(0.f, 0.f);
      const float2 c = (two && in_bounds(i0 + L, ext.in, kbInverseThetaIn)) ? F1[mp] : make_float2(0.f, 0.f);
      // F_{m,-m'} = sig F_{m m'}, column m+1: -sig; the phase e^{i pi (+-m')/N} rides on the
      // input chirp
      return (n < L) ? cadd(a, c) : cscale(csub(a, c), sig);
    };
    auto sink = [&](int k, float2 v) { buf[pidx(k)] = v; };
    bluestein<M, 1, false, true>(buf, tid, tw, tb, N, src, sink);
    __syncthreads();
    if (active) {
      // separate the two columns and write h[b][t][m mod N] with the phi phase e^{i pi m/N}
      const float2 e0 = tb.ph[m + N - 1], e1 = two ? tb.ph[m + 1 + N - 1] : e0;
      const int k0 = m >= 0 ? m : m + N, k1 = (m + 1) >= 0 ? m + 1 : m + 1 + N;
      float2* hb = h + (size_t)b * L * N;
      for (int t = tid; t < L; t += Geo<M>::T) {
        const float2 z = buf[pidx(t)], zr = buf[pidx(N - 1 - t)];
        const long long o = (hb - h) + (long long)t * N;
        if (two) {
          const float2 x0 = cscale(cadd(z, cscale(zr, sig)), 0.5f), x1 = cscale(csub(z, cscale(zr, sig)), 0.5f);
          if (in_bounds(o + k0, ext.out, kbInverseThetaOut)) hb[(size_t)t * N + k0] = cmul(x0, e0);
          if (in_bounds(o + k1, ext.out, kbInverseThetaOut)) hb[(size_t)t * N + k1] = cmul(x1, e1);
        } else if (in_bounds(o + k0, ext.out, kbInverseThetaOut)) {
          hb[(size_t)t * N + k0] = cmul(z, e0);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// rows along phi: inverse h -> f; forward f -> X[b][m][t] (scale 1/N for the forward transform)
// ---------------------------------------------------------------------------------------------
template <int M, int SIGN>
__global__ void __launch_bounds__(Geo<M>::THREADS, Geo<M>::MINB) phi_kernel(int L, int B, float scale, const float2* __restrict__ in,
                                                             float2* __restrict__ out, TorusTables tb, Ext ext) {
  float2* tw;
  float2* buf = setup_smem<M>(tb, &tw);
  const int Lp = L - 1, N = 2 * L - 1;
  const int tid = threadIdx.x % Geo<M>::T;
  const long long nrows = (long long)B * L;
  for (long long u0 = (long long)blockIdx.x * Geo<M>::G; u0 < nrows; u0 += (long long)gridDim.x * Geo<M>::G) {
    const long long u = u0 + threadIdx.x / Geo<M>::T;
    const bool active = u < nrows;
    const float2* x = in + (size_t)(active ? u : 0) * N;
    if (u + (long long)gridDim.x * Geo<M>::G < nrows)
      prefetch_l2(in + (size_t)(u + (long long)gridDim.x * Geo<M>::G) * N, (size_t)N * sizeof(float2), tid, Geo<M>::T);
    auto src = [&](int n) {
      return (active && in_bounds((long long)u * N + n, ext.in, kbPhiIn)) ? x[n] : make_float2(0.f, 0.f);
    };
    if constexpr (SIGN > 0) {
      float2* y = out + (size_t)(active ? u : 0) * N;
      auto sink = [&](int k, float2 v) {
        if (active && in_bounds((long long)u * N + k, ext.out, kbPhiOut)) y[k] = v;
      };
      bluestein<M, SIGN>(buf, tid, tw, tb, N, src, sink);
    } else {
      const int b = active ? (int)(u / L) : 0, t = active ? (int)(u % L) : 0;
      float2* Xb = out + (size_t)b * (N + 1) * L + 2 * t;
      auto sink = [&](int k, float2 v) {
        if (!active) return;
        const int mr = (k <= Lp ? k : k - N) + Lp;  // column m + Lp
        const size_t o = (size_t)(mr >> 1) * 2 * L + (mr & 1);
        if (in_bounds((Xb - out) + (long long)o, ext.out, kbPhiOut))
          Xb[o] = cscale(v, scale);  // e^{-i pi m/N} in the output chirp
      };
      bluestein<M, SIGN, true>(buf, tid, tw, tb, N, src, sink);
    }
    __syncthreads();
  }
}

// Element (b, m, m') of the forward projection's data tiles (the layout of the tensor-core
// contraction: tile (|m|, m' / 32) of 128-byte swizzled rows j = (m < 0) NC/2 + 2b + part, K = m'
// mod 32, the negative-m half carrying (-1)^{m'}): both parts of v, split.  The m = 0 tile's
// negative half and the padding rows b >= B are written as zeros by the passes of m = 0 and of
// the last field.
__device__ __forceinline__ void put_tile(const TileOut& to, int bg, int Bg, int mm, int mp, float2 v) {
  // field bg of Bg lies in slice bg / Bs, as field b of its B fields
  const int sl = bg / to.Bs, b = bg - sl * to.Bs, B = min(to.Bs, Bg - sl * to.Bs);
  const int am = mm < 0 ? -mm : mm, sign = mm < 0 ? 1 : 0;
  // a tile is one part (3xTF32: FP32 values) or two (split-BF16) of pb bytes in global memory
  const int pb = to.NC * 128, half = to.NC / 2, k = mp & 31, parts = to.mode == 2 ? 2 : 1;
  const size_t tb = (size_t)parts * pb;
  const long long tix = (long long)sl * (long long)(to.xslice / tb) + (long long)am * to.nC + (mp >> 5);
  uint8_t* tile = to.X + (size_t)sl * to.xslice + ((size_t)am * to.nC + (mp >> 5)) * tb;
  if (sign && (mp & 1)) v = make_float2(-v.x, -v.y);
  const bool tile_ok = in_bounds(tix, (long long)(to.xbytes / tb), kbPutTile);
  auto put = [&](int row, float x) {
    if (!tile_ok || !in_bounds(row, to.NC, kbPutTile)) return;
    if (to.mode == 2) tc::put_split<true>(tile, pb, row, k, x);
    else tc::put_split<false>(tile, pb, row, k, x);
  };
  put(sign * half + 2 * b, v.x);
  put(sign * half + 2 * b + 1, v.y);
  if (am == 0) {
    put(half + 2 * b, 0.f);
    put(half + 2 * b + 1, 0.f);
  }
  if (b == B - 1)
    for (int r = 2 * B; r < half; ++r) {
      put(sign * half + r, 0.f);
      if (am == 0) put(half + r, 0.f);
    }
}

// ---------------------------------------------------------------------------------------------
// forward theta analysis with the sin(theta) weight: X (pairs of columns) -> H[b][m][m'], or the
// projection's data tiles when to.mode != 0
// ---------------------------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(Geo<M>::THREADS, Geo<M>::MINB) forward_theta_kernel(int L, int s, int B, const float2* __restrict__ X,
                                                                       float2* __restrict__ H, TorusTables tb, TileOut to,
                                                                       Ext ext) {
  float2* tw;
  float2* buf = setup_smem<M>(tb, &tw);
  const int Lp = L - 1, N = 2 * L - 1;
  const int tid = threadIdx.x % Geo<M>::T;
  const long long npairs = (long long)B * L;
  for (long long u0 = (long long)blockIdx.x * Geo<M>::G; u0 < npairs; u0 += (long long)gridDim.x * Geo<M>::G) {
    const long long u = u0 + threadIdx.x / Geo<M>::T;
    const bool active = u < npairs;
    const int b = active ? (int)(u / L) : 0, p = active ? (int)(u % L) : 0;
    const int m = -Lp + 2 * p;
    const bool two = p < Lp;
    const bool odd0 = ((m + s) & 1) != 0;
    const float sig = odd0 ? -1.f : 1.f;
    const float4* Xp = (const float4*)(X + ((size_t)b * (N + 1) + 2 * p) * L);  // pair p: columns m, m + 1
    {
      const long long un = u + (long long)gridDim.x * Geo<M>::G;
      if (un < npairs)
        prefetch_l2(X + ((size_t)(un / L) * (N + 1) + 2 * (un % L)) * L, (size_t)L * sizeof(float4), tid, Geo<M>::T);
    }
    // extended samples of both columns on theta in [0, 2 pi): the odd one vanishes at theta = pi
    auto src = [&](int n) {
      if (!active) return make_float2(0.f, 0.f);
      const int t = n < L ? n : N - 1 - n;
      const bool ok = in_bounds(((const float2*)Xp - X) + 2LL * t + 1, ext.in, kbForwardThetaIn);
      const float4 ac = ok ? Xp[t] : make_float4(0.f, 0.f, 0.f, 0.f);
      float2 a = make_float2(ac.x, ac.y);
      float2 c = two ? make_float2(ac.z, ac.w) : make_float2(0.f, 0.f);
      if (t == Lp) {
        if (odd0) a = make_float2(0.f, 0.f);
        else c = make_float2(0.f, 0.f);
      }
      return (n < L) ? cadd(a, c) : cscale(csub(a, c), sig);
    };
    // Four FFTs of size M chained by fused passes: the theta DFT by Bluestein with centred
    // outputs (the kernel's spectrum khat_c puts F_{m''}, |m''| < L, at position m'' mod M), then
    // the circular convolution with the even weight, y = IFFT(FFT(F) * what), what = FFT(w_e)/M.
    // Between the DFT and the convolution F_{m''} takes its output chirp, the phase
    // e^{-i pi m''/N} and 1/N, and the positions L .. M - L (no frequency) become zeros.
    {
      auto in = [&](int n) {
        if (n >= N) return make_float2(0.f, 0.f);
        return cmul(src(n), __ldg(&tb.chirp[n]));
      };
      auto kmul = [&](int k, float2 v) { return cmul(v, __ldg(&tb.khat_c[k])); };
      auto fmul = [&](int k, float2 v) { return cmul(v, __ldg(&tb.chirp_c[k])); };
      auto wmul = [&](int k, float2 v) { return cmul(v, __ldg(&tb.what[k])); };
      auto cout = [&](int k, float2 v) { buf[pidx(k)] = v; };
      NoSrc none_in;
      NoSink none_out;
      constexpr int NP = Plan16<M>::NP;
      run_range<M, -1, 0, NP - 1, 1>(buf, tid, tw, in, none_out);
      boundary<M, -1, 1>(buf, tid, tw, kmul);
      run_range<M, 1, 1, NP - 1>(buf, tid, tw, none_in, none_out);
      boundary<M, 1, -1>(buf, tid, tw, fmul);
      run_range<M, -1, 1, NP - 1>(buf, tid, tw, none_in, none_out);
      boundary<M, -1, 1>(buf, tid, tw, wmul);
      run_range<M, 1, 1, NP>(buf, tid, tw, none_in, cout);
    }
    if (active) {
      // y[m'] = H'_m[m'] + H'_{m+1}[m'], y[-m'] = sig (H'_m[m'] - H'_{m+1}[m']); fold m' < 0:
      // H = (2 - delta_{m'0}) 2 pi H'.  Tiles: the last chunk's columns m' >= L are zeros.
      float2* H0 = to.mode ? nullptr : H + ((size_t)b * N + (m + Lp)) * L;
      float2* H1 = H0 + L;
      const float c2 = 6.28318530717958648f, c4 = 12.5663706143591730f;
      const int end = to.mode ? to.nC * 32 : L;
      for (int mp = tid; mp < end; mp += Geo<M>::T) {
        float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
        if (mp < L) {
          const float2 yp = buf[pidx(mp)], ym = buf[pidx((M - mp) & (M - 1))];
          const float c = mp == 0 ? c2 : c4;
          if (two) {
            v0 = cscale(cadd(yp, cscale(ym, sig)), 0.5f * c);
            v1 = cscale(csub(yp, cscale(ym, sig)), 0.5f * c);
          } else {
            v0 = cscale(yp, c);
          }
        }
        if (to.mode) {
          put_tile(to, b, B, m, mp, v0);
          if (two) put_tile(to, b, B, m + 1, mp, v1);
        } else {
          const long long o = (H0 - H) + mp;
          if (in_bounds(o, ext.out, kbForwardThetaOut)) H0[mp] = v0;
          if (two && in_bounds(o + L, ext.out, kbForwardThetaOut)) H1[mp] = v1;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// adjoint theta sums: X[b][m][t] (t < L, no extension) -> H[b][m][m'] = H'_{m'} + s_m H'_{-m'}
// ---------------------------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(Geo<M>::THREADS, Geo<M>::MINB) adjoint_theta_kernel(int L, int s, int B, const float2* __restrict__ X,
                                                                       float2* __restrict__ H, TorusTables tb, TileOut to,
                                                                       Ext ext) {
  float2* tw;
  float2* buf = setup_smem<M>(tb, &tw);
  const int Lp = L - 1, N = 2 * L - 1;
  const int tid = threadIdx.x % Geo<M>::T;
  const long long nrows = (long long)B * N;
  for (long long u0 = (long long)blockIdx.x * Geo<M>::G; u0 < nrows; u0 += (long long)gridDim.x * Geo<M>::G) {
    const long long u = u0 + threadIdx.x / Geo<M>::T;
    const bool active = u < nrows;
    const int mr = active ? (int)(u % N) : 0;  // column m + Lp of field u / N
    const int m = mr - Lp;
    const float2* x = X + ((size_t)(active ? u / N : 0) * (N + 1) + (mr & ~1)) * L + (mr & 1);
    {
      const long long un = u + (long long)gridDim.x * Geo<M>::G;
      if (un < nrows) {
        const int mrn = (int)(un % N);
        prefetch_l2(X + ((size_t)(un / N) * (N + 1) + (mrn & ~1)) * L, (size_t)L * sizeof(float4), tid, Geo<M>::T);
      }
    }
    auto src = [&](int n) {
      return (active && n < L && in_bounds((x - X) + 2LL * n, ext.in, kbAdjointThetaIn)) ? x[2 * n]
                                                                                         : make_float2(0.f, 0.f);
    };
    auto sink = [&](int k, float2 v) { buf[pidx(k)] = v; };  // H'_{m''} at bin k (phase in the chirp)
    bluestein<M, -1, true>(buf, tid, tw, tb, N, src, sink);
    __syncthreads();
    if (active) {
      const float sig = ((m + s) & 1) ? -1.f : 1.f;
      if (to.mode) {
        // the projection's data tiles (the last chunk's columns m' >= L are zeros)
        const int b = (int)(u / N);
        for (int mp = tid; mp < to.nC * 32; mp += Geo<M>::T) {
          float2 v = make_float2(0.f, 0.f);
          if (mp < L) {
            const float2 a = buf[pidx(mp)];
            v = mp == 0 ? a : cadd(a, cscale(buf[pidx(N - mp)], sig));
          }
          put_tile(to, b, B, m, mp, v);
        }
      } else {
        float2* Hr = H + (size_t)u * L;
        for (int mp = tid; mp < L; mp += Geo<M>::T) {
          const float2 a = buf[pidx(mp)];
          if (in_bounds(u * L + mp, ext.out, kbAdjointThetaOut)) Hr[mp] = mp == 0 ? a : cadd(a, cscale(buf[pidx(N - mp)], sig));
        }
      }
    }
    __syncthreads();
  }
}

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

template <class K>
cudaError_t set_smem(K kernel, int bytes) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e != cudaSuccess ? e : prefer_shared(kernel);
}

}  // namespace

struct TorusPlan {
  int L = 0, N = 0, M = 0;
  float2* buf = nullptr;  // chirp | khat_f | khat_i | what | twiddles (one allocation)
  TorusTables tb{};
  size_t bytes = 0;
  int smem = 0;
  int grid = 0;
};

cudaError_t torus_setup(TorusPlan** out, int L, const void* ph, int device) {
  *out = nullptr;
  const int N = 2 * L - 1;
  int M = 128;
  while (M < 2 * N - 1) M <<= 1;
  if (M > 8192) return cudaErrorInvalidValue;
  TorusPlan* p = new TorusPlan();
  p->L = L;
  p->N = N;
  p->M = M;
  const double pi = 3.14159265358979323846;
  // pass structure of the size-M FFT (mirrors Plan16)
  const int P16 = M >= 4096 ? 3 : M >= 256 ? 2 : 1, REST = M >> (4 * P16);
  const int NP = P16 + (REST > 1 ? 1 : 0);
  int TW = 0;
  for (int i = 1, ns = 16; i < NP; ++i, ns *= 16) TW += ((i < P16 ? 16 : REST) - 1) * ns;
  std::vector<float2> host((size_t)N + 3 * (size_t)M + (size_t)TW + (size_t)N + 2 * (size_t)M);
  float2* chirp = host.data();
  float2* kf = chirp + N;
  float2* ki = kf + M;
  float2* wh = ki + M;
  float2* tw = wh + M;
  float2* cph = tw + TW;
  float2* kc = cph + N;
  float2* cc = kc + M;
  for (int n = 0; n < N; ++n) {
    const long long r = ((long long)n * n) % (2LL * N);
    chirp[n] = make_float2((float)std::cos(-pi * r / N), (float)std::sin(-pi * r / N));
    // e^{-i pi n^2/N} e^{-i pi m/N} = e^{-i pi (n^2 + m)/N}, m = n or n - N, the angle reduced exactly
    const long long m = n <= L - 1 ? n : n - N;
    const long long rp = (((long long)n * n + m) % (2LL * N) + 2LL * N) % (2LL * N);
    cph[n] = make_float2((float)std::cos(-pi * rp / N), (float)std::sin(-pi * rp / N));
  }
  {
    float2* t = tw;
    for (int i = 1, ns = 16; i < NP; ++i, ns *= 16) {
      const int R = i < P16 ? 16 : REST;
      for (int r = 1; r < R; ++r)
        for (int j = 0; j < ns; ++j) {
          const double a = -2 * pi * (double)j * r / ((double)ns * R);
          *t++ = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    }
  }
  // output chirp of the centred forward DFT: F_m at m mod M with e^{-i pi (m^2 + m)/N}/N, zero
  // where no frequency sits
  for (int k = 0; k < M; ++k) {
    const long long m = k < L ? k : k > M - L ? (long long)k - M : 0;
    const bool in_band = k < L || k > M - L;
    const long long r = (((m * m + m) % (2LL * N)) + 2LL * N) % (2LL * N);
    cc[k] = in_band ? make_float2((float)(std::cos(-pi * r / N) / N), (float)(std::sin(-pi * r / N) / N))
                    : make_float2(0.f, 0.f);
  }
  // chirp kernel e^{+- i pi j^2/N} at j mod M: j in (-N, N) for outputs k in [0, N) (dir 0 forward,
  // 1 inverse); j in [-(N - 1) - (L - 1), L - 1] for the centred outputs |k| < L (dir 2), the same
  // count 2N - 1 <= M of distinct positions
  for (int dir = 0; dir < 3; ++dir) {
    std::vector<std::complex<double>> b(M, 0.0);
    const int jlo = dir == 2 ? -(N - 1) - (L - 1) : -(N - 1), jhi = dir == 2 ? L - 1 : N - 1;
    for (int j = jlo; j <= jhi; ++j) {
      const long long jj = (long long)j * j % (2LL * N);
      const double a = (dir == 1 ? -1.0 : 1.0) * pi * (double)jj / (double)N;
      b[((j % M) + M) % M] = std::complex<double>(std::cos(a), std::sin(a));
    }
    host_fft(b, -1);
    float2* dst = dir == 0 ? kf : dir == 1 ? ki : kc;
    for (int k = 0; k < M; ++k) dst[k] = make_float2((float)(b[k].real() / M), (float)(b[k].imag() / M));
  }
  {
    // w_e(p) = 2/(1-p^2) for even |p| <= 2(L-1), placed at p mod M (M >= 4L-3 > 4(L-1): no overlap)
    std::vector<std::complex<double>> w(M, 0.0);
    for (int q = -2 * (L - 1); q <= 2 * (L - 1); q += 2) w[(q + M) % M] = 2.0 / (1.0 - (double)q * q);
    host_fft(w, -1);
    for (int k = 0; k < M; ++k) wh[k] = make_float2((float)(w[k].real() / M), (float)(w[k].imag() / M));
  }
  cudaError_t e = dev_malloc(&p->buf, host.size() * sizeof(float2));
  if (e != cudaSuccess) {
    delete p;
    return e;
  }
  p->bytes = host.size() * sizeof(float2);
  e = cudaMemcpy(p->buf, host.data(), p->bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    torus_destroy(p);
    return e;
  }
  p->tb.chirp = p->buf;
  p->tb.khat_f = p->buf + N;
  p->tb.khat_i = p->buf + N + M;
  p->tb.what = p->buf + N + 2 * M;
  p->tb.tw = p->buf + N + 3 * M;
  p->tb.ph = (const float2*)ph;
  p->tb.chirp_ph = p->buf + N + 3 * M + TW;
  p->tb.khat_c = p->tb.chirp_ph + N;
  p->tb.chirp_c = p->tb.khat_c + M;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  p->grid = sms * 8;
#define SSHT_TP_ATTR(MM)                                                                               \
  if (M == MM) {                                                                                       \
    if (Plan16<MM>::TW != TW) {                                                                        \
      torus_destroy(p);                                                                                \
      return cudaErrorInvalidValue;                                                                    \
    }                                                                                                  \
    p->smem = Geo<MM>::SMEM;                                                                           \
    if ((e = set_smem(inverse_theta_kernel<MM>, p->smem)) != cudaSuccess ||                            \
        (e = set_smem(phi_kernel<MM, 1>, p->smem)) != cudaSuccess ||                                   \
        (e = set_smem(phi_kernel<MM, -1>, p->smem)) != cudaSuccess ||                                  \
        (e = set_smem(forward_theta_kernel<MM>, p->smem)) != cudaSuccess ||                            \
        (e = set_smem(adjoint_theta_kernel<MM>, p->smem)) != cudaSuccess) {                            \
      torus_destroy(p);                                                                                \
      return e;                                                                                        \
    }                                                                                                  \
  }
  SSHT_TP_ATTR(128) SSHT_TP_ATTR(256) SSHT_TP_ATTR(512) SSHT_TP_ATTR(1024) SSHT_TP_ATTR(2048)
  SSHT_TP_ATTR(4096) SSHT_TP_ATTR(8192)
#undef SSHT_TP_ATTR
  *out = p;
  return cudaSuccess;
}

void torus_destroy(TorusPlan* p) {
  if (!p) return;
  if (p->buf) cudaFree(p->buf);
  delete p;
}

size_t torus_bytes(const TorusPlan* p) { return p ? p->bytes : 0; }

// which: 0 inverse theta (F -> h), 1 inverse phi (h -> f), 2 forward phi (f -> X, scale 1/N),
// 3 adjoint phi (f -> X, no scale), 4 forward theta (X -> H), 5 adjoint theta (X -> H).
cudaError_t torus_pass(const TorusPlan* p, int which, int s, int B, const void* in, size_t in_bytes, void* out,
                       size_t out_bytes, cudaStream_t st, const TileOut* tiles) {
  const int L = p->L, M = p->M;
  const Ext ext{(long long)(in_bytes / sizeof(float2)), (long long)(out_bytes / sizeof(float2))};
  const TileOut to = ((which == 4 || which == 5) && tiles) ? *tiles : TileOut();
  const long long rows = (which == 1 || which == 2 || which == 3) ? (long long)B * L
                         : (which == 5)                            ? (long long)B * p->N
                                                                   : (long long)B * L;  // pairs
#define SSHT_TP_LAUNCH(MM)                                                                                   \
  if (M == MM) {                                                                                             \
    const long long need = (rows + Geo<MM>::G - 1) / Geo<MM>::G;                                            \
    const unsigned blocks = (unsigned)std::min<long long>(need, (long long)p->grid);                        \
    const dim3 thr(Geo<MM>::THREADS);                                                                        \
    const float2* I = (const float2*)in;                                                                     \
    float2* O = (float2*)out;                                                                                \
    switch (which) {                                                                                         \
      case 0: inverse_theta_kernel<MM><<<blocks, thr, p->smem, st>>>(L, s, B, I, O, p->tb, ext); break;     \
      case 1: phi_kernel<MM, 1><<<blocks, thr, p->smem, st>>>(L, B, 1.f, I, O, p->tb, ext); break;          \
      case 2: phi_kernel<MM, -1><<<blocks, thr, p->smem, st>>>(L, B, 1.f / (float)p->N, I, O, p->tb, ext); break; \
      case 3: phi_kernel<MM, -1><<<blocks, thr, p->smem, st>>>(L, B, 1.f, I, O, p->tb, ext); break;         \
      case 4: forward_theta_kernel<MM><<<blocks, thr, p->smem, st>>>(L, s, B, I, O, p->tb, to, ext); break; \
      case 5: adjoint_theta_kernel<MM><<<blocks, thr, p->smem, st>>>(L, s, B, I, O, p->tb, to, ext); break; \
      default: return cudaErrorInvalidValue;                                                                 \
    }                                                                                                        \
    return cudaGetLastError();                                                                               \
  }
  SSHT_TP_LAUNCH(128) SSHT_TP_LAUNCH(256) SSHT_TP_LAUNCH(512) SSHT_TP_LAUNCH(1024) SSHT_TP_LAUNCH(2048)
  SSHT_TP_LAUNCH(4096) SSHT_TP_LAUNCH(8192)
#undef SSHT_TP_LAUNCH
  return cudaErrorInvalidValue;
}

SSHT_BOUNDS_TU(torus_pass)

}  // namespace ssht
