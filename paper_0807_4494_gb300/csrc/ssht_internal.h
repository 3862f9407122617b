// Internal declarations of libssht (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/ssht.h"

namespace ssht {

// Every kernel of the library asks for the largest shared-memory carveout of the SM's unified
// L1 / shared array.  CTAs of different kernels share an SM only under one carveout, and the
// recursion (one CTA per SM for the whole sweep) is meant to share its SMs with the kernels of
// the other stream.
template <class K>
inline cudaError_t prefer_shared(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// Device status word bits (latched by kernels, read by ssht_plan_check).
enum : int { kStatusOk = 0, kStatusBarrierTimeout = 1 };

// Sizes derived from the exclusive band-limit L.
struct Dims {
  int L;   // exclusive band-limit
  int Lp;  // L - 1, the paper's inclusive band-limit
  int N;   // 2L - 1 torus samples per axis
  int M;   // length of the zero-padded weight convolution, >= 4L - 3
};

// Records the message returned by ssht_last_error() and returns code.
int set_last_error(int code, const char* msg);

// Every device allocation of the library goes through here (cudaMalloc), so that the test hook
// ssht_debug_fail_allocation can make a chosen one fail as if the device were out of memory.
cudaError_t dev_malloc(void** ptr, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T** ptr, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(ptr), bytes);
}

inline size_t delta_offset(long long l) { return (size_t)(l * (l + 1) * (2 * l + 1) / 6); }
inline size_t tri(long long l) { return (size_t)(l * (l + 1) / 2); }

// ---------------------------------------------------------------------------
// Delta recursion (delta.cu)
// ---------------------------------------------------------------------------
// How the Delta table is made: the three-term relation in m' (delta_column.cu, the default) or
// the Risbo recursion the paper uses (delta.cu).
enum : int { kDeltaColumn = 0, kDeltaRisbo = 1 };

struct DeltaWork {
  int method = kDeltaColumn;
  double* table = nullptr;        // quadrant table, delta_offset(L) doubles
  double* slab[2] = {nullptr, nullptr};  // padded octant slabs (rows 0..L, columns -1..m+1)
  double* sqrt_tab = nullptr;     // sqrt(k), k = 0 .. 2L + 2
  unsigned int* barrier = nullptr;  // grid barrier counter
  int* status = nullptr;          // latched status word
  int blocks = 0;                 // cooperative grid size
  int threads = 0;
  size_t smem = 0;
  size_t bytes = 0;   // device memory held (table, slabs, tables, words)
  int4* part = nullptr;   // per step and CTA: owned rows and the CTAs waited for
  size_t bytes_part = 0;
  long long cap = 0;  // shared-memory doubles per CTA
  int2* tasks = nullptr;  // column method: (degree, column block) tasks, longest first
  int ntasks = 0;
};

cudaError_t delta_setup(DeltaWork& w, int L, int device, int method = kDeltaColumn);
void delta_free(DeltaWork& w);
// wait_ns: spin limit of the Risbo recursion's waits (the column recursion has none).
constexpr long long kDefaultWaitNs = 1000000000ll;
cudaError_t delta_run(const DeltaWork& w, int L, cudaStream_t st, long long wait_ns = kDefaultWaitNs);
// The column method's setup and launch (delta_column.cu); delta_setup / delta_run dispatch.
cudaError_t column_setup(DeltaWork& w, int L, int device);
cudaError_t column_run(const DeltaWork& w, int L, cudaStream_t st);
// U[l][m'] = sqrt((2l+1)/4pi) Delta^l_{m',-s}, l < L, 0 <= m' <= l, at tri(l) + m'; Uf is the
// same in FP32 (rounded to nearest).
cudaError_t delta_spin_column(const double* table, int L, int s, double* U, float* Uf, cudaStream_t st);

// ---------------------------------------------------------------------------
// SIMT contractions (contract_simt.cu); T is double or float
// ---------------------------------------------------------------------------
// Inverse: half = 0 writes the theta-DFT input E[b][m + Lp][k], k = m' mod N, of the extended,
// phase-shifted F (eqn fourier_coeff, eqn Ffourier_sym, eqn idft_spatial phase); half = 1 writes
// the half rows F[b][m + Lp][m'], 0 <= m' < L, without phases (the torus passes' input).
template <typename T>
cudaError_t contract_inverse_simt(const Dims& d, int s, int B, const double* table, const double* U,
                                  const void* flm, size_t flm_bytes, void* E, size_t e_bytes, const double2* ph, int half,
                                  cudaStream_t st);
// Projection: flm[b][l*l+l+m] = (-1)^s i^{m+s} c_l sum_{m'>=0} Delta_{m'm} Delta_{m',-s} H[b][m+Lp][m']
template <typename T>
cudaError_t contract_project_simt(const Dims& d, int s, int B, const double* table, const double* U,
                                  const void* H, size_t h_bytes, void* flm, size_t flm_bytes, cudaStream_t st);

// The paper's triangular forward (triangular.cu), FP64: Fk = theta-DFT bins of the extended
// columns [B][N][N] (no phase, no 1/N), flm [B][L*L] double2.
cudaError_t triangular_solve(const Dims& d, int s, int B, const double* table, const double* U, const void* Fk,
                             const double2* ph, void* flm, cudaStream_t st);

// Real spin-0 fields two to a complex field (real.cu); T is double or float.  flm: [nreal][L*L]
// complex, f: [nreal][L][2L-1] real; rc, rg: the complex pairs ([ceil(nreal/2)][...]).
template <typename T> cudaError_t real_pack_coeffs(int L, int nreal, const void* flm, void* rc, cudaStream_t st);
template <typename T> cudaError_t real_pack_grid(int L, int nreal, const void* f, void* rg, cudaStream_t st);
template <typename T> cudaError_t real_unpack_grid(int L, int nreal, const void* rg, void* f, cudaStream_t st);
template <typename T> cudaError_t real_unpack_coeffs(int L, int nreal, const void* rc, void* flm, cudaStream_t st);
// Spin pairs (real.cu): c [B][L*L] spin-s coefficients -> out [B][2][L*L] (spin s, then spin -s of
// the conjugate field); in [B][2][L*L] -> c [B][L*L] (the spin-s halves).
template <typename T> cudaError_t pair_expand(int L, int s, int B, const void* c, void* out, cudaStream_t st);
template <typename T> cudaError_t pair_gather(int L, int B, const void* in, void* c, cudaStream_t st);
// Kernel attributes of the packing kernels (on the current device).
cudaError_t real_setup();

// ---------------------------------------------------------------------------
// Tensor-core contractions (contract_tc.cu), 3xTF32 or split-BF16
// ---------------------------------------------------------------------------
struct TcPlan;
// The contraction's tunable shape: fields per GEMM launch (the N tile: 2 x 2 x slice real columns,
// padded to 16), pipeline depth (stages of A and data tiles in shared memory), and the order of the
// work items (inverse: 0 grouped by m, 1 longest first; forward: 0 longest first, 1 grouped by m).
struct TcConfig {
  int slice = 64;
  int stages = 2;
  int inv_order = 0;
  int fwd_order = 0;
};
// bf16 = 0: 3xTF32 split products; bf16 = 1: split-BF16 (three parts, six products).  Any batch:
// the fields run in slices of at most 64.
cudaError_t tc_setup(TcPlan** out, int L, int s, int B, int bf16, int device);
bool tc_config_fits(const TcPlan* p, const TcConfig& c);  // within the device's shared memory
cudaError_t tc_configure(TcPlan* p, const TcConfig& c);    // reallocates the data tiles if needed
TcConfig tc_config(const TcPlan* p);
void tc_destroy(TcPlan* p);
size_t tc_bytes(const TcPlan* p);
// Pack the A operand (U_l[m'] Delta^l_{m'm} in FP32, then split) of one direction from the FP64
// table and the FP32 copy of U.
cudaError_t tc_pack_a(TcPlan* p, int forward, const double* table, const float* U, cudaStream_t st, int* launches);
// Pack the inverse's data operand V from flm (float2 [B][L*L]); the forward's and the adjoint's
// data tiles come from their theta passes (TileOut).
cudaError_t tc_pack_data(TcPlan* p, const void* src, cudaStream_t st, int* launches);
// The contraction: forward = 0 writes the half rows F (float2 [B][N][L], m' >= 0) of the inverse;
// forward = 1 writes flm (float2 [B][L*L]).  Timeouts set bit 2 of *status.
cudaError_t tc_gemm(TcPlan* p, int forward, void* out, const void* ph, int* status, long long wait_ns, cudaStream_t st,
                    int* launches);
// Where the forward theta pass writes the projection's data tiles directly (in place of H and
// tc_pack_data): the tile array, its column count NC, chunks per m nC, and the split form
// (mode 1: 3xTF32, 2: split-BF16; 0: no tiles, H is written).
struct TileOut {
  uint8_t* X = nullptr;
  int NC = 0, nC = 0, mode = 0;
  int Bs = 64;        // fields per slice; slice z of the fields has its tiles at X + z * xslice
  size_t xslice = 0;
  size_t xbytes = 0;  // the whole tile array (index checks)
};
TileOut tc_forward_tiles(const TcPlan* p);
// Where the recursion can write the A operand itself (3xTF32 plans): the forward tile array and
// its per-m tile index base; A is null for split-BF16 plans (their A comes from tc_pack_a).
struct ATiles {
  uint8_t* A = nullptr;
  const long long* abase = nullptr;
  long long ntiles = 0;  // tiles in A (index checks)
};
ATiles tc_a_tiles(const TcPlan* p);
// The column recursion writing the A tiles of a 3xTF32 plan directly (no FP64 table):
// A_m[l][m'] = Uf_l[m'] Delta^l_{m'm} in FP32, one value an entry, by the rescaled relation whose
// tables lt holds (delta_column.cu).
struct LaneTables;
cudaError_t column_run_tiles(const DeltaWork& w, const LaneTables& lt, int L, const float* Uf, ATiles t,
                             cudaStream_t st);
// The inverse contraction's A tiles (rows m', K = l) of a 3xTF32 plan: the tile array and, per
// (m, row block i), the index from which chunk kc's tile is ibase[m * nI + i] + kc.
struct InvTiles {
  uint8_t* A = nullptr;
  const long long* ibase = nullptr;
  int nI = 0;
  int nC = 0;
  long long ntiles = 0;  // tiles in A (index checks)
};
InvTiles tc_inverse_tiles(const TcPlan* p);
// Plan-time tables of the recursion with one lane per degree, which writes the inverse's tiles
// directly (delta_column.cu): coefficients a(l, m'), b(l, m'), first rows (mantissa, exponent), U
// transposed, in the triangle layout [r][l] (l >= r); its tasks (column m, chunk kc of 32 degrees).
// Plan-time tables of the tile-writing recursions (3xTF32 plans): the rescaled relation's
// alpha(l, m') and p(l, m') degree-major (l(l+1)/2 + m') and in the triangle layout [m'][l], the
// first rows and U transposed (delta_column.cu).
struct LaneTables {
  double* alc = nullptr;
  float* pc = nullptr;
  double* alT = nullptr;
  float* pT = nullptr;
  double* t1m = nullptr;
  int* t1e = nullptr;
  float* ufT = nullptr;
  long long* ab2 = nullptr;  // per M: the forward tile base less the row blocks below M's own
  int2* tasks = nullptr;
  int ntasks = 0;
  int blocks = 0;      // grid of the degree-lane recursion
  int col_blocks = 0;  // grid of the column recursion writing the forward tiles
  size_t bytes = 0;
};
// Needs the column DeltaWork of the plan (its sqrt tables) and U (FP32) on the device; synchronises.
cudaError_t lane_tables_setup(LaneTables& t, const DeltaWork& w, int L, int s, const float* Uf, int nC,
                              const long long* abase);
void lane_tables_free(LaneTables& t);
cudaError_t column_run_inverse_tiles(const DeltaWork& w, const LaneTables& t, int L, int s, InvTiles it,
                                     cudaStream_t st);

// ---------------------------------------------------------------------------
// Fused torus passes of FP32 plans (torus_pass.cu)
// ---------------------------------------------------------------------------
// Odd-length DFTs along theta and phi (Bluestein in shared memory) with the extension, phases, sin(theta) weight convolution and transpositions folded in.  Layouts (float2):
// F half rows [B][N][L] (m + Lp, m' >= 0), h [B][L][N], f [B][L][N], X [B][(N+1)/2][L][2] (columns
// m + Lp = 2p + j by pairs), H [B][N][L].
struct TorusPlan;
cudaError_t torus_setup(TorusPlan** out, int L, const void* ph, int device);
void torus_destroy(TorusPlan* p);
size_t torus_bytes(const TorusPlan* p);
// which: 0 inverse theta (F -> h), 1 inverse phi (h -> f), 2 forward phi (f -> X, scale 1/N),
// 3 adjoint phi (f -> X), 4 forward theta with the weight convolution (X -> H), 5 adjoint theta (X -> H).
// which = 4 with tiles (mode != 0): the data tiles of the forward projection instead of H.
// in_bytes / out_bytes: the extents of the buffers (the index checks of bounds-checked builds).
cudaError_t torus_pass(const TorusPlan* p, int which, int s, int B, const void* in, size_t in_bytes, void* out,
                       size_t out_bytes, cudaStream_t st, const TileOut* tiles = nullptr);

// ---------------------------------------------------------------------------
// Torus kernels (torus.cu)
// ---------------------------------------------------------------------------
// g[b][m+Lp][t] (theta-synthesis output, N per row) -> h[b][t][m mod N] * e^{i pi m / N}, t < L.
template <typename T>
cudaError_t inv_theta_to_phi(const Dims& d, int B, const void* g, void* h, const void* ph, cudaStream_t st);
// X[b][t][k] (phi-DFT of the samples) -> ext[b][m+Lp][t'] (theta-DFT input).
// mode 0: forward (per-m parity extension, factor e^{-i pi m/N}/N);
// mode 1: adjoint (zero rings t' >= L, factor e^{-i pi m/N}).
template <typename T>
cudaError_t fwd_phi_to_theta(const Dims& d, int s, int B, int mode, const void* X, void* ext, const void* ph,
                             cudaStream_t st);
// Fk[b][m+Lp][k'] (theta-DFT) -> zero-padded conv input cx[b][m+Lp][j], j = m'' mod M,
// value F_{m m''} = Fk[k'(m'')] e^{-i pi m''/N} / N.
template <typename T>
cudaError_t fwd_theta_to_conv(const Dims& d, int B, const void* Fk, void* cx, const void* ph, cudaStream_t st);
// Pointwise product of the conv spectrum with the weight spectrum (real kernel, length M).
template <typename T>
cudaError_t conv_multiply(const Dims& d, int B, void* cx, const void* khat, cudaStream_t st);
// Conv output y[b][m+Lp][j] -> H[b][m+Lp][m'] = c_{m'} y[m'] / M, m' in [0, Lp], c_0 = 2pi, else 4pi.
template <typename T>
cudaError_t conv_to_project(const Dims& d, int B, const void* y, void* H, cudaStream_t st);
// Adjoint: Fk (theta-DFT of the zero-padded rings) -> folded H[b][m+Lp][m'], m' in [0, Lp]:
// H'_{m m'} + (-1)^{m+s} H'_{m,-m'} (m' > 0), H'_{m 0} (m' = 0), H'_{m m'} = Fk[k'(m')] e^{-i pi m'/N}.
template <typename T>
cudaError_t adj_theta_fold(const Dims& d, int s, int B, const void* Fk, void* H, const void* ph, cudaStream_t st);
// Weight kernel kappa[p mod M] = w_e(p) = 2/(1-p^2) for even |p| <= 2Lp (0 otherwise); its FFT is
// the spectrum used by conv_multiply.  The phase table ph[k + N - 1] = e^{i pi k/N}, |k| < N, is
// complex in the element precision T (double2 or float2).
template <typename T>
cudaError_t make_weight_kernel(const Dims& d, void* kappa, cudaStream_t st);


// ---------------------------------------------------------------------------
// Index checks of bounds-checked builds (bounds.cuh): each translation unit's record, copied out
// and cleared.
// ---------------------------------------------------------------------------
struct BoundsRecord;
cudaError_t bounds_take_torus_pass(BoundsRecord* r);
cudaError_t bounds_take_contract_tc(BoundsRecord* r);
cudaError_t bounds_take_delta_column(BoundsRecord* r);
cudaError_t bounds_take_real(BoundsRecord* r);
cudaError_t bounds_take_contract_simt(BoundsRecord* r);

}  // namespace ssht
