// C ABI of libssht (declared in include/ssht.h): plans, workspaces, the order of the
// stages of each transform, host-pointer staging and error reporting.
#include "ssht_internal.h"
#include "bounds.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace ssht;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

}  // namespace

namespace ssht {
int set_last_error(int code, const char* msg) { return fail(code, msg); }

namespace {
std::atomic<long long> g_alloc_countdown{0};
}

cudaError_t dev_malloc(void** ptr, size_t bytes) {
  long long n = g_alloc_countdown.load();
  while (n > 0 && !g_alloc_countdown.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 1) {  // this is the chosen allocation: fail it like an exhausted device
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}
}  // namespace ssht

namespace {

const char* cufft_name(cufftResult r) {
  switch (r) {
    case CUFFT_SUCCESS: return "CUFFT_SUCCESS";
    case CUFFT_INVALID_PLAN: return "CUFFT_INVALID_PLAN";
    case CUFFT_ALLOC_FAILED: return "CUFFT_ALLOC_FAILED";
    case CUFFT_INVALID_VALUE: return "CUFFT_INVALID_VALUE";
    case CUFFT_INTERNAL_ERROR: return "CUFFT_INTERNAL_ERROR";
    case CUFFT_EXEC_FAILED: return "CUFFT_EXEC_FAILED";
    case CUFFT_SETUP_FAILED: return "CUFFT_SETUP_FAILED";
    case CUFFT_INVALID_SIZE: return "CUFFT_INVALID_SIZE";
    default: return "cuFFT error";
  }
}

#define SSHT_CUDA(x, what)                                                                         \
  do {                                                                                             \
    cudaError_t e_ = (x);                                                                          \
    if (e_ != cudaSuccess) {                                                                       \
      return fail(e_ == cudaErrorMemoryAllocation ? SSHT_ENOMEM : SSHT_ECUDA,                      \
                  std::string(what) + ": " + cudaGetErrorString(e_));                              \
    }                                                                                              \
  } while (0)

#define SSHT_FFT(x, what)                                                                          \
  do {                                                                                             \
    cufftResult r_ = (x);                                                                          \
    if (r_ != CUFFT_SUCCESS) {                                                                     \
      return fail(r_ == CUFFT_ALLOC_FAILED ? SSHT_ENOMEM : SSHT_ECUDA,                             \
                  std::string(what) + ": " + cufft_name(r_));                                      \
    }                                                                                              \
  } while (0)

// Smallest 2^a 3^b 5^c 7^d >= n (a length cuFFT handles with its fast radices).
int good_fft_size(int n) {
  for (int m = n > 1 ? n : 1;; ++m) {
    int r = m;
    for (int p : {2, 3, 5, 7})
      while (r % p == 0) r /= p;
    if (r == 1) return m;
  }
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct ssht_plan_s {
  int device = 0;
  Dims d{};
  int s = 0, B = 0, precision = 0, delta_mode = 0;
  bool f64 = true;
  size_t elem = 16;  // bytes per complex element of the I/O and workspaces
  DeltaWork delta;
  double* U = nullptr;
  float* Uf = nullptr;  // U in FP32 (tensor-core operand packing)
  void* W1 = nullptr;
  void* W2 = nullptr;
  size_t w_bytes = 0;  // each of W1, W2
  void* W3 = nullptr;
  void* khat = nullptr;
  void* ph = nullptr;       // phase table, element precision
  double2* ph64 = nullptr;  // phase table, FP64
  cufftHandle fft_phi = 0, fft_theta = 0, fft_conv = 0;
  bool have_phi = false, have_theta = false, have_conv = false;
  void* stage_in = nullptr;
  size_t stage_in_bytes = 0;
  void* stage_out = nullptr;
  size_t stage_out_bytes = 0;
  bool delta_ready = false;
  bool u_fixed = false;  // U / Uf made once at creation (3xTF32 plans with the recursion writing the A tiles)
  long long wait_ns = kDefaultWaitNs;  // spin limit of the device-side waits
  LaneTables lane;  // tables of the recursion that writes the inverse's A tiles (3xTF32, own recursion)
  size_t bytes = 0;
  TcPlan* tc = nullptr;    // tensor-core contraction (precisions SSHT_TF32X3, SSHT_BF16X6)
  TorusPlan* torus = nullptr;  // fused torus passes of FP32 plans (FP64 plans: cuFFT Z2Z + glue)
  // The Delta recursion (and the A packing) of a call runs on a second stream, forked from the
  // caller's stream at the start of the call and joined before the contraction, so that the
  // Delta-independent work of the call (the torus stage of forward/adjoint, data packing) runs
  // beside it.
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool join_pending = false;
  // A plan of a group shares the Delta table of its band-limit with the group's other plans:
  // the group runs the recursion (recorded by delta_event), the plan only its spin column.
  bool delta_shared = false;
  cudaEvent_t delta_event = nullptr;
  // What the next call's recursion and packing (on aux) must wait for, instead of the whole of
  // the previous calls: ev_free after the last kernel on a caller's stream that read the Delta
  // table or U (SIMT contractions, the triangular solve, the table copy; the tensor-core path reads
  // them only on aux, in order), and ev_free_a[dir] after the tensor-core contraction that read the
  // A tiles of that direction.  Each is usable only within the capture sequence it was recorded in
  // (0 = not capturing); otherwise, or before the first record, the call forks from the caller's
  // stream as a whole.
  cudaEvent_t ev_free = nullptr;
  bool free_valid = false;
  unsigned long long free_capture = 0;
  cudaEvent_t ev_free_a[2] = {nullptr, nullptr};
  bool afree_valid[2] = {false, false};
  unsigned long long afree_capture[2] = {0, 0};
  // profiling: events bracketing each stage, folded into per-stage totals on read
  struct Ev {
    int stage;
    int lane;  // 0: the call's stream, 1: the plan's second stream
    cudaEvent_t a, b;
  };
  bool prof = false;
  std::vector<Ev> evs;
  double prof_ms[SSHT_NUM_STAGES] = {};
  long long prof_n[SSHT_NUM_STAGES] = {};
  long long launches = 0;

  // Real spin-0 fields (SSHT_FLAG_REAL): nreal caller fields ride two to a complex field; B is
  // the number of complex fields the transforms see, rc / rg their coefficients and samples.
  bool real = false;
  int nreal = 0;
  void* rc = nullptr;
  void* rg = nullptr;

  // Spin pairs (SSHT_FLAG_SPIN_PAIR): coefficients [B][2][L*L], spin s then spin -s of the
  // conjugate field; rc holds the spin-s halves.
  bool pair = false;

  // bytes of the caller's buffers
  size_t coeff_bytes() const { return (size_t)(real ? nreal : B) * d.L * d.L * elem * (pair ? 2 : 1); }
  size_t grid_bytes() const { return real ? (size_t)nreal * d.L * d.N * (elem / 2) : (size_t)B * d.L * d.N * elem; }
  size_t pair_coeff_bytes() const { return (size_t)B * d.L * d.L * elem; }
  size_t pair_grid_bytes() const { return (size_t)B * d.L * d.N * elem; }
};

namespace {

void fold_events(ssht_plan_t p) {
  for (auto& e : p->evs) {
    float ms = 0.f;
    if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      p->prof_ms[e.stage] += ms;
      p->prof_n[e.stage] += 1;
    }
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  p->evs.clear();
}

// Brackets one stage with events on the call's stream while profiling is enabled.
struct StageScope {
  ssht_plan_t p;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageScope(ssht_plan_t p_, int stage_, cudaStream_t st_) : p(p_), stage(stage_), st(st_) {
    if (p->prof && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, st);
  }
  ~StageScope() {
    if (!a) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    cudaEventRecord(b, st);
    p->evs.push_back({stage, st == p->aux ? 1 : 0, a, b});
    if (p->evs.size() > 8192) fold_events(p);
  }
};

int dalloc(ssht_plan_t p, void** ptr, size_t bytes, const char* what) {
  cudaError_t e = dev_malloc(ptr, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(SSHT_ENOMEM, std::string("cudaMalloc ") + what + " (" + std::to_string(bytes) + " bytes): " +
                                 cudaGetErrorString(e));
  }
  p->bytes += bytes;
  return 0;
}

int exec_fft(const ssht_plan_t p, cufftHandle h, void* in, void* out, int dir, cudaStream_t st) {
  StageScope sc(p, SSHT_STAGE_FFT, st);
  if (p->f64) {
    SSHT_FFT(cufftExecZ2Z(h, (cufftDoubleComplex*)in, (cufftDoubleComplex*)out, dir), "cufftExecZ2Z");
  } else {
    SSHT_FFT(cufftExecC2C(h, (cufftComplex*)in, (cufftComplex*)out, dir), "cufftExecC2C");
  }
  return 0;
}

int run_dft(ssht_plan_t p, cufftHandle h, int sign, void* in, void* out, cudaStream_t st) {
  return exec_fft(p, h, in, out, sign < 0 ? CUFFT_FORWARD : CUFFT_INVERSE, st);
}

// One fused torus pass of an FP32 plan (DFT along theta or phi with its glue), timed as FFT work.
// in / out: a plan workspace (W1, W2) or a grid of the plan's B complex fields.
int run_torus(ssht_plan_t p, int which, const void* in, void* out, cudaStream_t st) {
  StageScope sc(p, SSHT_STAGE_FFT, st);
  const size_t grid = p->pair_grid_bytes();
  const size_t ib = (in == p->W1 || in == p->W2) ? p->w_bytes : grid;
  const size_t ob = (out == p->W1 || out == p->W2) ? p->w_bytes : grid;
  SSHT_CUDA(torus_pass(p->torus, which, p->s, p->B, in, ib, out, ob, st), "torus pass");
  p->launches += 1;
  return 0;
}

int make_fft(ssht_plan_t p, cufftHandle* h, bool* have, int n, size_t batch, const char* what) {
  if (batch > (size_t)0x7fffffff) return fail(SSHT_EUNSUPPORTED, std::string(what) + ": batch too large");
  int nn = n;
  SSHT_FFT(cufftPlanMany(h, 1, &nn, nullptr, 1, n, nullptr, 1, n, p->f64 ? CUFFT_Z2Z : CUFFT_C2C, (int)batch), what);
  *have = true;
  size_t ws = 0;
  if (cufftGetSize(*h, &ws) == CUFFT_SUCCESS) p->bytes += ws;
  return 0;
}

int set_streams(ssht_plan_t p, cudaStream_t st) {
  if (p->have_phi) SSHT_FFT(cufftSetStream(p->fft_phi, st), "cufftSetStream");
  if (p->have_theta) SSHT_FFT(cufftSetStream(p->fft_theta, st), "cufftSetStream");
  if (p->have_conv) SSHT_FFT(cufftSetStream(p->fft_conv, st), "cufftSetStream");
  return 0;
}

int pack_a(ssht_plan_t p, int forward, cudaStream_t st);

int run_delta(ssht_plan_t p, cudaStream_t st) {
  StageScope sc(p, SSHT_STAGE_DELTA, st);
  if (!p->delta_shared) {
    SSHT_CUDA(delta_run(p->delta, p->d.L, st, p->wait_ns), "Delta recursion launch");
    p->launches += 1;
  }
  if (!p->u_fixed) {
    SSHT_CUDA(delta_spin_column(p->delta.table, p->d.L, p->s, p->U, p->Uf, st), "spin column launch");
    p->launches += 1;
  }
  return 0;
}

// 3xTF32 plans that run their own column recursion make the contraction's A tiles in the
// recursion itself (no FP64 table, no packing): the forward's tiles (rows l, K = m') with one lane
// per column, the inverse's (rows m', K = l) with one lane per degree.  U, the spin column, and the
// degree-lane recursion's tables are made once at plan creation.
bool tiles_direct(const ssht_plan_s* p) {
  return p->tc && tc_a_tiles(p->tc).A && !p->delta_shared && p->delta.method == kDeltaColumn;
}

// Delta and the contraction's A operand of one direction, on st.
int make_operands(ssht_plan_t p, int forward, cudaStream_t st) {
  if (tiles_direct(p)) {
    StageScope sc(p, forward ? SSHT_STAGE_DELTA : SSHT_STAGE_DELTA_INVERSE, st);
    if (forward)
      SSHT_CUDA(column_run_tiles(p->delta, p->lane, p->d.L, p->Uf, tc_a_tiles(p->tc), st), "recursion into the A tiles");
    else
      SSHT_CUDA(column_run_inverse_tiles(p->delta, p->lane, p->d.L, p->s, tc_inverse_tiles(p->tc), st),
                "recursion into the inverse's A tiles");
    p->launches += 1;
    return 0;
  }
  int rc = run_delta(p, st);
  if (rc) return rc;
  return p->tc ? pack_a(p, forward, st) : 0;
}

int pack_a(ssht_plan_t p, int forward, cudaStream_t st) {
  StageScope sc(p, SSHT_STAGE_PACK, st);
  int n = 0;
  SSHT_CUDA(tc_pack_a(p->tc, forward, p->delta.table, p->Uf, st, &n), "tensor-core operand packing");
  p->launches += n;
  return 0;
}

int ensure_delta(ssht_plan_t p, cudaStream_t st) {
  if (p->delta_mode == SSHT_DELTA_CACHE && p->delta_ready) return 0;
  int rc = run_delta(p, st);
  if (rc) return rc;
  if (p->delta_mode == SSHT_DELTA_CACHE) p->delta_ready = true;
  return 0;
}

// Start making Delta (and, for the tensor-core path, the packed A operand of one direction) on
// the plan's second stream, after everything already queued on st; join_operands makes st wait.
unsigned long long capture_id(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  unsigned long long id = 0;
  if (cudaStreamGetCaptureInfo(st, &cs, &id) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return cs == cudaStreamCaptureStatusActive ? id : 0;
}

// After the last reader of the table, U and the A tiles in a call.
int mark_free(ssht_plan_t p, cudaStream_t st) {
  SSHT_CUDA(cudaEventRecord(p->ev_free, st), "operands-free event");
  p->free_valid = true;
  p->free_capture = capture_id(st);
  return 0;
}

// After the tensor-core contraction of one direction: the A tiles of that direction are free.
int mark_free_a(ssht_plan_t p, int forward, cudaStream_t st) {
  SSHT_CUDA(cudaEventRecord(p->ev_free_a[forward], st), "A-tiles-free event");
  p->afree_valid[forward] = true;
  p->afree_capture[forward] = capture_id(st);
  return 0;
}

// The inverse's A tiles of a plan whose recursions write them (3xTF32) are made as soon as the
// previous inverse contraction has read them, without waiting for the forward contraction in
// between: the degree-lane recursion then runs beside the forward's torus passes instead of beside
// the next call's data packing (GB300, L = 1024, B = 64: 11.995 ms a step against 12.095).
#ifndef SSHT_INVERSE_OPERANDS_EARLY
#define SSHT_INVERSE_OPERANDS_EARLY 1
#endif

int begin_operands(ssht_plan_t p, int forward, cudaStream_t st) {
  if (p->delta_mode == SSHT_DELTA_CACHE && p->delta_ready) return 0;
  const unsigned long long cap = capture_id(st);
  // the previous readers of what the aux work overwrites, if they are known
  const bool table_ok = !p->free_valid || p->free_capture == cap;
  const bool a_ok = !p->tc || !p->afree_valid[forward] || p->afree_capture[forward] == cap;
  const bool any = p->free_valid || (p->tc && p->afree_valid[forward]);
  if (table_ok && a_ok && any) {
    // only those readers: the rest of the previous calls (e.g. the inverse's torus stage) may
    // still be running while this call's recursion starts
    if (p->free_valid) SSHT_CUDA(cudaStreamWaitEvent(p->aux, p->ev_free, 0), "operands-free wait");
    if (p->tc && p->afree_valid[forward]) SSHT_CUDA(cudaStreamWaitEvent(p->aux, p->ev_free_a[forward], 0), "A-free wait");
    // ... and the other direction's contraction: it cannot share an SM with the recursion, so
    // queued behind a running recursion it would wait for the whole sweep, while run first
    // (about 1 ms) it lets the torus passes that follow it overlap the recursion (not for the
    // inverse's tiles of a 3xTF32 plan, see above)
    const bool early = SSHT_INVERSE_OPERANDS_EARLY && !forward && tiles_direct(p);
    if (p->tc && !early && p->afree_valid[1 - forward] && p->afree_capture[1 - forward] == cap)
      SSHT_CUDA(cudaStreamWaitEvent(p->aux, p->ev_free_a[1 - forward], 0), "other contraction wait");
  } else {
    SSHT_CUDA(cudaEventRecord(p->ev_fork, st), "fork event");
    SSHT_CUDA(cudaStreamWaitEvent(p->aux, p->ev_fork, 0), "fork wait");
  }
  if (p->delta_shared && p->delta_event) SSHT_CUDA(cudaStreamWaitEvent(p->aux, p->delta_event, 0), "shared Delta wait");
  int rc = make_operands(p, forward, p->aux);
  if (rc) return rc;
  SSHT_CUDA(cudaEventRecord(p->ev_join, p->aux), "join event");
  p->join_pending = true;
  return 0;
}

int join_operands(ssht_plan_t p, cudaStream_t st) {
  if (!p->join_pending) return 0;
  p->join_pending = false;
  SSHT_CUDA(cudaStreamWaitEvent(st, p->ev_join, 0), "join wait");
  return 0;
}

int tc_pack(ssht_plan_t p, const void* src, cudaStream_t st) {
  int n = 0;
  StageScope sc(p, SSHT_STAGE_PACK, st);
  SSHT_CUDA(tc_pack_data(p->tc, src, st, &n), "tensor-core data packing");
  p->launches += n;
  return 0;
}

int tc_multiply(ssht_plan_t p, int forward, void* dst, cudaStream_t st) {
  int n = 0;
  StageScope sc(p, forward ? SSHT_STAGE_PROJECT : SSHT_STAGE_INVERSE, st);
  SSHT_CUDA(tc_gemm(p->tc, forward, dst, p->ph, p->delta.status, p->wait_ns, st, &n), "tensor-core contraction");
  p->launches += n;
  return 0;
}

// Tensor-core forward / adjoint after the phi pass (in W2): the theta pass `which` (4 forward, 5
// adjoint) writes the projection's data tiles itself (no H, no data packing), then the projection.
int theta_to_tiles(ssht_plan_t p, int which, void* flm, cudaStream_t st) {
  int rc;
  const TileOut tiles = tc_forward_tiles(p->tc);
  {
    StageScope sc(p, SSHT_STAGE_FFT, st);
    SSHT_CUDA(torus_pass(p->torus, which, p->s, p->B, p->W2, p->w_bytes, nullptr, 0, st, &tiles), "torus pass");
    p->launches += 1;
  }
  if ((rc = join_operands(p, st)) || (rc = tc_multiply(p, 1, flm, st))) return rc;
  return mark_free_a(p, 1, st);
}

// The SIMT projection of forward / adjoint from the folded torus sums H (in W), after the join
// (tensor-core plans take theta_to_tiles).
template <typename T>
int project(ssht_plan_t p, const void* H, void* flm, cudaStream_t st) {
  int rc;
  if ((rc = join_operands(p, st))) return rc;
  {
    StageScope sc(p, SSHT_STAGE_PROJECT, st);
    SSHT_CUDA(contract_project_simt<T>(p->d, p->s, p->B, p->delta.table, p->U, H, p->w_bytes, flm, p->pair_coeff_bytes(), st),
              "projection");
    p->launches += 1;
  }
  return mark_free(p, st);
}

int check_device(ssht_plan_t p) {
  int cur = -1;
  SSHT_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
  if (cur != p->device)
    return fail(SSHT_EINVAL, "plan was created on device " + std::to_string(p->device) + " but device " +
                                 std::to_string(cur) + " is current");
  return 0;
}

int stage_buffer(ssht_plan_t p, void** buf, size_t* have, size_t need, const char* what) {
  if (*have >= need) return 0;
  if (*buf) {
    cudaFree(*buf);
    p->bytes -= *have;
    *buf = nullptr;
    *have = 0;
  }
  int rc = dalloc(p, buf, need, what);
  if (rc) return rc;
  *have = need;
  return 0;
}

// Resolve input/output pointers: host buffers go through plan-owned staging memory.
struct IO {
  const void* in_dev;
  void* out_dev;
  void* out_host;
  size_t out_bytes;
};

// A host input is copied to plan-owned device memory by the copy engines (cudaMemcpyAsync on the
// call's stream), not read in place by the first kernel over the host link: a kernel reading host
// memory holds its SMs for the whole transfer, while the copy engines leave them to the work of
// other streams (the plan's own recursion on its second stream, or another request's kernels).
int io_begin(ssht_plan_t p, const void* in, size_t in_bytes, void* out, size_t out_bytes, cudaStream_t st, IO* io) {
  if (!in || !out) return fail(SSHT_EINVAL, "null data pointer");
  io->out_host = nullptr;
  io->out_bytes = out_bytes;
  if (is_device_pointer(in)) {
    io->in_dev = in;
  } else {
    int rc = stage_buffer(p, &p->stage_in, &p->stage_in_bytes, in_bytes, "input staging");
    if (rc) return rc;
    SSHT_CUDA(cudaMemcpyAsync(p->stage_in, in, in_bytes, cudaMemcpyHostToDevice, st), "input copy to device");
    io->in_dev = p->stage_in;
  }
  if (is_device_pointer(out)) {
    io->out_dev = out;
  } else {
    int rc = stage_buffer(p, &p->stage_out, &p->stage_out_bytes, out_bytes, "output staging");
    if (rc) return rc;
    io->out_dev = p->stage_out;
    io->out_host = out;
  }
  return 0;
}

int io_end(ssht_plan_t p, const IO& io, cudaStream_t st) {
  (void)p;
  if (io.out_host) {
    SSHT_CUDA(cudaMemcpyAsync(io.out_host, io.out_dev, io.out_bytes, cudaMemcpyDeviceToHost, st),
              "output copy to host");
    SSHT_CUDA(cudaStreamSynchronize(st), "stream synchronize");
  }
  SSHT_CUDA(cudaGetLastError(), "kernel launch");
  return 0;
}

template <typename T>
int inverse_impl(ssht_plan_t p, const void* flm, void* f, cudaStream_t st) {
  const Dims& d = p->d;
  int rc = begin_operands(p, 0, st);
  if (rc) return rc;
  if (p->tc) {
    if ((rc = tc_pack(p, flm, st)) || (rc = join_operands(p, st)) || (rc = tc_multiply(p, 0, p->W1, st)) ||
        (rc = mark_free_a(p, 0, st)))
      return rc;
  } else {
    if ((rc = join_operands(p, st))) return rc;
    StageScope sc(p, SSHT_STAGE_INVERSE, st);
    SSHT_CUDA(contract_inverse_simt<T>(d, p->s, p->B, p->delta.table, p->U, flm, p->pair_coeff_bytes(), p->W1, p->w_bytes,
                                       p->ph64, p->torus ? 1 : 0, st),
              "inverse contraction");
    p->launches += 1;
  }
  if (!p->tc && (rc = mark_free(p, st))) return rc;
  if (p->torus) {
    if ((rc = run_torus(p, 0, p->W1, p->W2, st))) return rc;
    return run_torus(p, 1, p->W2, f, st);
  }
  rc = run_dft(p, p->fft_theta, +1, p->W1, p->W2, st);
  if (rc) return rc;
  {
    StageScope sc(p, SSHT_STAGE_TORUS, st);
    SSHT_CUDA(inv_theta_to_phi<T>(d, p->B, p->W2, p->W1, p->ph, st), "theta-to-phi transpose");
    p->launches += 1;
  }
  return run_dft(p, p->fft_phi, +1, p->W1, f, st);
}

// Shared front of the forward transform (mode 0) and the adjoint (mode 1): phi DFT,
// extension (or zero rings) into the theta-DFT input, theta DFT in place in W1.
template <typename T>
int analysis_front(ssht_plan_t p, const void* f, int mode, cudaStream_t st) {
  const Dims& d = p->d;
  int rc = run_dft(p, p->fft_phi, -1, const_cast<void*>(f), p->W2, st);
  if (rc) return rc;
  {
    StageScope sc(p, SSHT_STAGE_TORUS, st);
    SSHT_CUDA(fwd_phi_to_theta<T>(d, p->s, p->B, mode, p->W2, p->W1, p->ph, st), "phi-to-theta extension");
    p->launches += 1;
  }
  return run_dft(p, p->fft_theta, -1, p->W1, p->W1, st);
}

template <typename T>
int forward_impl(ssht_plan_t p, const void* f, void* flm, cudaStream_t st) {
  const Dims& d = p->d;
  int rc = begin_operands(p, 1, st);
  if (rc) return rc;
  if (p->torus) {
    if ((rc = run_torus(p, 2, f, p->W2, st))) return rc;
    if (p->tc) return theta_to_tiles(p, 4, flm, st);
    if ((rc = run_torus(p, 4, p->W2, p->W1, st))) return rc;
    return project<T>(p, p->W1, flm, st);
  }
  rc = analysis_front<T>(p, f, 0, st);
  if (rc) return rc;
  {
    StageScope sc(p, SSHT_STAGE_TORUS, st);
    SSHT_CUDA(fwd_theta_to_conv<T>(d, p->B, p->W1, p->W3, p->ph, st), "weight convolution input");
    p->launches += 1;
  }
  if ((rc = exec_fft(p, p->fft_conv, p->W3, p->W3, CUFFT_FORWARD, st))) return rc;
  {
    StageScope sc(p, SSHT_STAGE_TORUS, st);
    SSHT_CUDA(conv_multiply<T>(d, p->B, p->W3, p->khat, st), "weight convolution product");
    p->launches += 1;
  }
  if ((rc = exec_fft(p, p->fft_conv, p->W3, p->W3, CUFFT_INVERSE, st))) return rc;
  {
    StageScope sc(p, SSHT_STAGE_TORUS, st);
    SSHT_CUDA(conv_to_project<T>(d, p->B, p->W3, p->W1, st), "weight convolution output");
    p->launches += 1;
  }
  return project<T>(p, p->W1, flm, st);
}

template <typename T>
int adjoint_impl(ssht_plan_t p, const void* g, void* flm, cudaStream_t st) {
  const Dims& d = p->d;
  int rc = begin_operands(p, 1, st);
  if (rc) return rc;
  if (p->torus) {
    if ((rc = run_torus(p, 3, g, p->W2, st))) return rc;
    if (p->tc) return theta_to_tiles(p, 5, flm, st);
    if ((rc = run_torus(p, 5, p->W2, p->W1, st))) return rc;
    return project<T>(p, p->W1, flm, st);
  }
  rc = analysis_front<T>(p, g, 1, st);
  if (rc) return rc;
  {
    StageScope sc(p, SSHT_STAGE_TORUS, st);
    SSHT_CUDA(adj_theta_fold<T>(d, p->s, p->B, p->W1, p->W2, p->ph, st), "adjoint fold");
    p->launches += 1;
  }
  return project<T>(p, p->W2, flm, st);
}

// Real spin-0 fields, two to a complex field: which = 0 inverse, 1 forward, 2 adjoint.
template <typename T>
int real_call(ssht_plan_t p, int which, const void* in, void* out, cudaStream_t st) {
  const int L = p->d.L;
  int rc;
  {
    StageScope sc(p, SSHT_STAGE_PACK, st);
    if (which == 0) SSHT_CUDA(real_pack_coeffs<T>(L, p->nreal, in, p->rc, st), "real-field packing");
    else SSHT_CUDA(real_pack_grid<T>(L, p->nreal, in, p->rg, st), "real-field packing");
    p->launches += 1;
  }
  if (which == 0) rc = inverse_impl<T>(p, p->rc, p->rg, st);
  else if (which == 1) rc = forward_impl<T>(p, p->rg, p->rc, st);
  else rc = adjoint_impl<T>(p, p->rg, p->rc, st);
  if (rc) return rc;
  StageScope sc(p, SSHT_STAGE_PACK, st);
  if (which == 0) SSHT_CUDA(real_unpack_grid<T>(L, p->nreal, p->rg, out, st), "real-field unpacking");
  else SSHT_CUDA(real_unpack_coeffs<T>(L, p->nreal, p->rc, out, st), "real-field unpacking");
  p->launches += 1;
  return 0;
}

// Spin pairs: which = 0 inverse (from the spin-s halves), 1 forward, 2 adjoint (one spin-s
// transform, then the spin -s coefficients of the conjugate field by the conjugate symmetry).
template <typename T>
int pair_call(ssht_plan_t p, int which, const void* in, void* out, cudaStream_t st) {
  const int L = p->d.L;
  int rc;
  if (which == 0) {
    {
      StageScope sc(p, SSHT_STAGE_PACK, st);
      SSHT_CUDA(pair_gather<T>(L, p->B, in, p->rc, st), "spin-pair gather");
      p->launches += 1;
    }
    return inverse_impl<T>(p, p->rc, out, st);
  }
  rc = which == 1 ? forward_impl<T>(p, in, p->rc, st) : adjoint_impl<T>(p, in, p->rc, st);
  if (rc) return rc;
  StageScope sc(p, SSHT_STAGE_PACK, st);
  SSHT_CUDA(pair_expand<T>(L, p->s, p->B, p->rc, out, st), "spin-pair expansion");
  p->launches += 1;
  return 0;
}

// ---------------------------------------------------------------------------------------------
// Tile tuning of the tensor-core contraction (SSHT_FLAG_TUNE, and the tuned buckets of groups):
// every shape candidate -- fields per GEMM launch, pipeline depth, work order -- is timed on the
// plan's own operands (inverse + forward contractions, CUDA events) and the fastest kept.  With
// SSHT_TUNE_CACHE naming a file, choices are looked up there first and stored after tuning, one
// JSON object per line: {"key": "L=1024 s=2 B=64 tf32x3", "slice": 64, "stages": 2, ...}.
// ---------------------------------------------------------------------------------------------
std::string tune_key(const ssht_plan_s* p) {
  return "L=" + std::to_string(p->d.L) + " s=" + std::to_string(p->s) + " B=" + std::to_string(p->B) +
         (p->precision == SSHT_BF16X6 ? " bf16x6" : " tf32x3");
}

bool tune_cache_lookup(const std::string& key, TcConfig* c) {
  const char* path = std::getenv("SSHT_TUNE_CACHE");
  if (!path || !*path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  const std::string want = "{\"key\": \"" + key + "\",";
  while (std::fgets(line, sizeof line, f)) {
    if (std::strncmp(line, want.c_str(), want.size()) != 0) continue;
    TcConfig t;
    if (std::sscanf(line + want.size(), " \"slice\": %d, \"stages\": %d, \"inv_order\": %d, \"fwd_order\": %d", &t.slice,
                    &t.stages, &t.inv_order, &t.fwd_order) == 4) {
      *c = t;
      found = true;  // the last entry of a key wins
    }
  }
  std::fclose(f);
  return found;
}

void tune_cache_store(const std::string& key, const TcConfig& c, float ms) {
  const char* path = std::getenv("SSHT_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "{\"key\": \"%s\", \"slice\": %d, \"stages\": %d, \"inv_order\": %d, \"fwd_order\": %d, \"ms\": %.4f}\n",
               key.c_str(), c.slice, c.stages, c.inv_order, c.fwd_order, ms);
  std::fclose(f);
}

int make_operands(ssht_plan_t p, int forward, cudaStream_t st);

// Mean milliseconds of one inverse + one forward contraction of the plan's current shape.
int time_contractions(ssht_plan_t p, cudaStream_t st, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SSHT_CUDA(cudaEventCreate(&e0), "tuning event");
  SSHT_CUDA(cudaEventCreate(&e1), "tuning event");
  int n = 0, rc = 0;
  for (int it = 0; it < 4 && !rc; ++it) {
    if (it == 1) cudaEventRecord(e0, st);
    cudaError_t e = tc_gemm(p->tc, 0, p->W1, p->ph, p->delta.status, p->wait_ns, st, &n);
    if (e == cudaSuccess) e = tc_gemm(p->tc, 1, p->W2, p->ph, p->delta.status, p->wait_ns, st, &n);
    if (e != cudaSuccess) rc = fail(SSHT_ECUDA, std::string("tuning contraction: ") + cudaGetErrorString(e));
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  *ms = t / 3.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int tune_tiles(ssht_plan_t p) {
  if (!p->tc) return 0;
  TcConfig best = tc_config(p->tc);
  const std::string key = tune_key(p);
  if (tune_cache_lookup(key, &best) && tc_config_fits(p->tc, best)) {
    SSHT_CUDA(tc_configure(p->tc, best), "tile configuration");
    return 0;
  }
  cudaStream_t st = nullptr;
  SSHT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "tuning stream");
  auto done = [&](int rc) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
  };
  int rc = 0;
  // the operands of both directions, once (the data tiles' values do not change the timing)
  if ((rc = make_operands(p, 0, st)) || (rc = make_operands(p, 1, st))) return done(rc);
  float best_ms = 0.f;
  bool have = false;
  auto trial = [&](const TcConfig& c) {
    if (!tc_config_fits(p->tc, c)) return 0;
    cudaError_t e = tc_configure(p->tc, c);
    if (e != cudaSuccess) return fail(SSHT_ECUDA, std::string("tile configuration: ") + cudaGetErrorString(e));
    float ms = 0.f;
    int r = time_contractions(p, st, &ms);
    if (r) return r;
    if (!have || ms < best_ms) {
      best_ms = ms;
      best = c;
      have = true;
    }
    return 0;
  };
  std::vector<int> slices;
  for (int sl : {64, 32, 16}) {
    const int bs = std::min(sl, p->B);
    if (std::find(slices.begin(), slices.end(), bs) == slices.end()) slices.push_back(bs);
  }
  for (int sl : slices)
    for (int stg = 2; stg <= 4; ++stg) {
      TcConfig c;
      c.slice = sl;
      c.stages = stg;
      if ((rc = trial(c))) return done(rc);
    }
  const TcConfig shape = best;
  for (int io = 0; io < 2; ++io)
    for (int fo = 0; fo < 2; ++fo) {
      if (io == shape.inv_order && fo == shape.fwd_order) continue;
      TcConfig c = shape;
      c.inv_order = io;
      c.fwd_order = fo;
      if ((rc = trial(c))) return done(rc);
    }
  cudaError_t e = tc_configure(p->tc, best);
  if (e != cudaSuccess) return done(fail(SSHT_ECUDA, std::string("tile configuration: ") + cudaGetErrorString(e)));
  tune_cache_store(key, best, best_ms);
  return done(0);
}

void release(ssht_plan_t p) {
  if (!p) return;
  cudaDeviceSynchronize();
  for (auto& e : p->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  if (p->tc) tc_destroy(p->tc);
  if (p->torus) torus_destroy(p->torus);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->ev_free) cudaEventDestroy(p->ev_free);
  for (cudaEvent_t e : p->ev_free_a)
    if (e) cudaEventDestroy(e);
  if (p->aux) cudaStreamDestroy(p->aux);
  if (p->have_phi) cufftDestroy(p->fft_phi);
  if (p->have_theta) cufftDestroy(p->fft_theta);
  if (p->have_conv) cufftDestroy(p->fft_conv);
  if (!p->delta_shared) delta_free(p->delta);
  lane_tables_free(p->lane);
  void* ptrs[] = {p->U, p->Uf, p->W1, p->W2, p->W3, p->khat, p->ph, p->ph64, p->stage_in, p->stage_out, p->rc, p->rg};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete p;
}

int create(ssht_plan_t* out, const ssht_plan_desc* desc, const DeltaWork* shared = nullptr) {
  if (!out || !desc) return fail(SSHT_EINVAL, "null argument");
  *out = nullptr;
  const int L = desc->L, s = desc->s, nfields = desc->batch;
  if (L < 1 || L > 2048) return fail(SSHT_EINVAL, "band-limit L must be in [1, 2048]");
  if (s <= -L || s >= L) return fail(SSHT_EINVAL, "spin must satisfy |s| < L");
  if (nfields < 1 || nfields > 65535) return fail(SSHT_EINVAL, "batch must be in [1, 65535]");
  if ((desc->flags & ~(SSHT_FLAG_REAL | SSHT_FLAG_RISBO | SSHT_FLAG_TUNE | SSHT_FLAG_SPIN_PAIR)) != 0)
    return fail(SSHT_EINVAL, "unknown flags");
  const bool pair = (desc->flags & SSHT_FLAG_SPIN_PAIR) != 0;
  if (pair && (desc->flags & SSHT_FLAG_REAL)) return fail(SSHT_EINVAL, "SSHT_FLAG_SPIN_PAIR and SSHT_FLAG_REAL exclude each other");
  if (pair && shared) return fail(SSHT_EINVAL, "groups take single fields, not spin pairs");
  const bool real = (desc->flags & SSHT_FLAG_REAL) != 0;
  if (real && s != 0) return fail(SSHT_EINVAL, "real fields (SSHT_FLAG_REAL) need spin 0");
  if (real && shared) return fail(SSHT_EINVAL, "groups take complex fields only");
  const int B = real ? (nfields + 1) / 2 : nfields;  // complex fields the transforms see
  if (desc->delta_mode != SSHT_DELTA_RECOMPUTE && desc->delta_mode != SSHT_DELTA_CACHE)
    return fail(SSHT_EINVAL, "unknown Delta mode");
  if (desc->precision != SSHT_FP64 && desc->precision != SSHT_FP32 && desc->precision != SSHT_TF32X3 &&
      desc->precision != SSHT_BF16X6)
    return fail(SSHT_EINVAL, "unknown precision");

  ssht_plan_t p = new (std::nothrow) ssht_plan_s();
  if (!p) return fail(SSHT_ENOMEM, "host allocation of the plan");
  int rc = 0;
  cudaError_t ce = cudaGetDevice(&p->device);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->ev_free, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->ev_free_a[0], cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&p->ev_free_a[1], cudaEventDisableTiming);
  if (ce != cudaSuccess) {
    release(p);
    return fail(SSHT_ECUDA, std::string("plan stream/event setup: ") + cudaGetErrorString(ce));
  }
  p->d.L = L;
  p->d.Lp = L - 1;
  p->d.N = 2 * L - 1;
  p->d.M = good_fft_size(4 * L - 3);
  p->s = s;
  p->B = B;
  p->precision = desc->precision;
  p->delta_mode = desc->delta_mode;
  p->real = real;
  p->nreal = real ? nfields : 0;
  p->pair = pair;
  p->f64 = desc->precision == SSHT_FP64;
  p->elem = p->f64 ? 16 : 8;
  const Dims& d = p->d;

  auto bail = [&](int code) {
    release(p);
    return code;
  };
  if (shared) {
    p->delta = *shared;
    p->delta_shared = true;
  } else {
    ce = delta_setup(p->delta, L, p->device, (desc->flags & SSHT_FLAG_RISBO) ? kDeltaRisbo : kDeltaColumn);
    if (ce != cudaSuccess) {
      release(p);
      return fail(ce == cudaErrorMemoryAllocation ? SSHT_ENOMEM : SSHT_ECUDA,
                  std::string("Delta recursion setup: ") + cudaGetErrorString(ce));
    }
    p->bytes += p->delta.bytes;
  }
  if (real && (ce = real_setup()) != cudaSuccess) {
    release(p);
    return fail(SSHT_ECUDA, std::string("real-field kernel attributes: ") + cudaGetErrorString(ce));
  }
  if ((rc = dalloc(p, (void**)&p->U, tri(L) * sizeof(double), "spin column"))) return bail(rc);
  if ((rc = dalloc(p, (void**)&p->Uf, tri(L) * sizeof(float), "spin column (FP32)"))) return bail(rc);
  // FP64: full N x N torus rows and an M-point convolution buffer; FP32 (fused torus passes): half
  // rows of N x L only, plus one row a field for the column pairs of the phi pass's output.
  const size_t torus = (size_t)B * (p->f64 ? (size_t)d.N * d.N : (size_t)(d.N + 1) * d.L) * p->elem;
  if (pair && (rc = dalloc(p, &p->rc, (size_t)B * L * L * p->elem, "spin-pair coefficients"))) return bail(rc);
  if ((real || pair) && (ce = real_setup()) != cudaSuccess) {
    release(p);
    return fail(SSHT_ECUDA, std::string("packing kernel attributes: ") + cudaGetErrorString(ce));
  }
  if (real) {
    if ((rc = dalloc(p, &p->rc, p->pair_coeff_bytes(), "real-field pair coefficients"))) return bail(rc);
    if ((rc = dalloc(p, &p->rg, p->pair_grid_bytes(), "real-field pair samples"))) return bail(rc);
  }
  if ((rc = dalloc(p, &p->W1, torus, "torus workspace 1"))) return bail(rc);
  if ((rc = dalloc(p, &p->W2, torus, "torus workspace 2"))) return bail(rc);
  p->w_bytes = torus;
  if (p->f64) {
    if ((rc = dalloc(p, &p->W3, (size_t)B * d.N * d.M * p->elem, "convolution workspace"))) return bail(rc);
    if ((rc = dalloc(p, &p->khat, (size_t)d.M * p->elem, "weight spectrum"))) return bail(rc);
  }
  if ((rc = dalloc(p, &p->ph, (size_t)(2 * d.N - 1) * p->elem, "phase table"))) return bail(rc);
  if ((rc = dalloc(p, (void**)&p->ph64, (size_t)(2 * d.N - 1) * sizeof(double2), "phase table"))) return bail(rc);

  // Phase table e^{i pi k / N}, |k| < N, computed in FP64 on the host.
  {
    std::vector<double2> h(2 * d.N - 1);
    std::vector<float2> hf(2 * d.N - 1);
    const double pi = 3.14159265358979323846;
    for (int k = -(d.N - 1); k <= d.N - 1; ++k) {
      // reduce the angle to [-pi/2, pi/2]-ish before cos/sin for accuracy: k/N in (-1, 1)
      const double a = pi * (double)k / (double)d.N;
      h[k + d.N - 1] = make_double2(std::cos(a), std::sin(a));
      hf[k + d.N - 1] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    ce = cudaMemcpy(p->ph64, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess)
      ce = cudaMemcpy(p->ph, p->f64 ? (const void*)h.data() : (const void*)hf.data(), h.size() * p->elem,
                      cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      release(p);
      return fail(SSHT_ECUDA, std::string("phase table upload: ") + cudaGetErrorString(ce));
    }
  }
  if (p->f64) {
    if ((rc = make_fft(p, &p->fft_phi, &p->have_phi, d.N, (size_t)B * d.L, "cuFFT phi plan"))) return bail(rc);
    if ((rc = make_fft(p, &p->fft_theta, &p->have_theta, d.N, (size_t)B * d.N, "cuFFT theta plan"))) return bail(rc);
    if ((rc = make_fft(p, &p->fft_conv, &p->have_conv, d.M, (size_t)B * d.N, "cuFFT convolution plan")))
      return bail(rc);
    // Weight spectrum: FFT of the even part of w(p) = int_0^pi sin(t) e^{ipt} dt.
    cufftHandle k1;
    int nn = d.M;
    cufftResult r = cufftPlan1d(&k1, nn, CUFFT_Z2Z, 1);
    if (r != CUFFT_SUCCESS) {
      release(p);
      return fail(SSHT_ECUDA, std::string("cuFFT weight plan: ") + cufft_name(r));
    }
    ce = make_weight_kernel<double>(d, p->khat, 0);
    if (ce == cudaSuccess) r = cufftExecZ2Z(k1, (cufftDoubleComplex*)p->khat, (cufftDoubleComplex*)p->khat, CUFFT_FORWARD);
    cudaError_t se = cudaDeviceSynchronize();
    cufftDestroy(k1);
    if (ce != cudaSuccess || r != CUFFT_SUCCESS || se != cudaSuccess) {
      release(p);
      return fail(SSHT_ECUDA, "weight spectrum setup failed");
    }
  } else {
    ce = torus_setup(&p->torus, L, p->ph, p->device);
    if (ce != cudaSuccess) {
      release(p);
      return fail(ce == cudaErrorMemoryAllocation ? SSHT_ENOMEM : SSHT_ECUDA,
                  std::string("torus pass setup: ") + cudaGetErrorString(ce));
    }
    p->bytes += torus_bytes(p->torus);
  }
  if (desc->precision == SSHT_TF32X3 || desc->precision == SSHT_BF16X6) {
    ce = tc_setup(&p->tc, L, s, B, desc->precision == SSHT_BF16X6 ? 1 : 0, p->device);
    if (ce != cudaSuccess) {
      release(p);
      return fail(ce == cudaErrorMemoryAllocation ? SSHT_ENOMEM : SSHT_ECUDA,
                  std::string("tensor-core plan: ") + cudaGetErrorString(ce));
    }
    p->bytes += tc_bytes(p->tc);
  }
  if (tiles_direct(p)) {
    // the spin column once: the table of one sweep, then U from it
    if ((rc = run_delta(p, 0))) return bail(rc);
    p->u_fixed = true;
    // the calls' recursions run on the plan's non-blocking stream: U must be complete first
    ce = cudaDeviceSynchronize();
    if (ce == cudaSuccess)
      ce = lane_tables_setup(p->lane, p->delta, L, s, p->Uf, tc_inverse_tiles(p->tc).nC, tc_a_tiles(p->tc).abase);
    if (ce != cudaSuccess) {
      release(p);
      return fail(ce == cudaErrorMemoryAllocation ? SSHT_ENOMEM : SSHT_ECUDA,
                  std::string("spin column and recursion tables: ") + cudaGetErrorString(ce));
    }
    p->bytes += p->lane.bytes;
  }
  if (p->delta_mode == SSHT_DELTA_CACHE) {
    if (tiles_direct(p)) {
      if ((rc = make_operands(p, 0, 0)) || (rc = make_operands(p, 1, 0))) return bail(rc);
    } else {
      if ((rc = run_delta(p, 0))) return bail(rc);
      if (p->tc && ((rc = pack_a(p, 0, 0)) || (rc = pack_a(p, 1, 0)))) return bail(rc);
    }
    ce = cudaDeviceSynchronize();
    if (ce != cudaSuccess) {
      release(p);
      return fail(SSHT_ECUDA, std::string("Delta recursion: ") + cudaGetErrorString(ce));
    }
    int st = 0;
    cudaMemcpy(&st, p->delta.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (st != 0) {
      release(p);
      return fail(SSHT_ETIMEOUT, "Delta recursion grid barrier timed out");
    }
    p->delta_ready = true;
  }
  if ((desc->flags & SSHT_FLAG_TUNE) && (rc = tune_tiles(p))) return bail(rc);
  *out = p;
  g_last_error.clear();
  return SSHT_OK;
}

}  // namespace

extern "C" {

int ssht_plan(ssht_plan_t* out, int L, int s, int batch) {
  ssht_plan_desc d{L, s, batch, SSHT_FP64, SSHT_DELTA_RECOMPUTE, 0};
  return create(out, &d);
}

int ssht_plan_ex(ssht_plan_t* out, const ssht_plan_desc* desc) { return create(out, desc); }

int ssht_plan_destroy(ssht_plan_t plan) {
  release(plan);
  return SSHT_OK;
}

int ssht_plan_workspace_bytes(ssht_plan_t plan, size_t* bytes) {
  if (!plan || !bytes) return fail(SSHT_EINVAL, "null argument");
  *bytes = plan->bytes;
  return SSHT_OK;
}

int ssht_inverse(ssht_plan_t p, const void* flm, void* f, void* stream) {
  if (!p) return fail(SSHT_EINVAL, "null plan");
  int rc = check_device(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = set_streams(p, st))) return rc;
  IO io;
  if ((rc = io_begin(p, flm, p->coeff_bytes(), f, p->grid_bytes(), st, &io))) return rc;
  if (p->real)
    rc = p->f64 ? real_call<double>(p, 0, io.in_dev, io.out_dev, st) : real_call<float>(p, 0, io.in_dev, io.out_dev, st);
  else if (p->pair)
    rc = p->f64 ? pair_call<double>(p, 0, io.in_dev, io.out_dev, st) : pair_call<float>(p, 0, io.in_dev, io.out_dev, st);
  else
    rc = p->f64 ? inverse_impl<double>(p, io.in_dev, io.out_dev, st) : inverse_impl<float>(p, io.in_dev, io.out_dev, st);
  if (rc) return rc;
  return io_end(p, io, st);
}

int ssht_forward(ssht_plan_t p, const void* f, void* flm, void* stream) {
  if (!p) return fail(SSHT_EINVAL, "null plan");
  int rc = check_device(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = set_streams(p, st))) return rc;
  IO io;
  if ((rc = io_begin(p, f, p->grid_bytes(), flm, p->coeff_bytes(), st, &io))) return rc;
  if (p->real)
    rc = p->f64 ? real_call<double>(p, 1, io.in_dev, io.out_dev, st) : real_call<float>(p, 1, io.in_dev, io.out_dev, st);
  else if (p->pair)
    rc = p->f64 ? pair_call<double>(p, 1, io.in_dev, io.out_dev, st) : pair_call<float>(p, 1, io.in_dev, io.out_dev, st);
  else
    rc = p->f64 ? forward_impl<double>(p, io.in_dev, io.out_dev, st) : forward_impl<float>(p, io.in_dev, io.out_dev, st);
  if (rc) return rc;
  return io_end(p, io, st);
}

int ssht_adjoint(ssht_plan_t p, const void* g, void* flm, void* stream) {
  if (!p) return fail(SSHT_EINVAL, "null plan");
  int rc = check_device(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = set_streams(p, st))) return rc;
  IO io;
  if ((rc = io_begin(p, g, p->grid_bytes(), flm, p->coeff_bytes(), st, &io))) return rc;
  if (p->real)
    rc = p->f64 ? real_call<double>(p, 2, io.in_dev, io.out_dev, st) : real_call<float>(p, 2, io.in_dev, io.out_dev, st);
  else if (p->pair)
    rc = p->f64 ? pair_call<double>(p, 2, io.in_dev, io.out_dev, st) : pair_call<float>(p, 2, io.in_dev, io.out_dev, st);
  else
    rc = p->f64 ? adjoint_impl<double>(p, io.in_dev, io.out_dev, st) : adjoint_impl<float>(p, io.in_dev, io.out_dev, st);
  if (rc) return rc;
  return io_end(p, io, st);
}

int ssht_forward_triangular(ssht_plan_t p, const void* f, void* flm, void* stream) {
  if (!p) return fail(SSHT_EINVAL, "null plan");
  if (!p->f64) return fail(SSHT_EUNSUPPORTED, "the triangular forward is built for FP64 plans only");
  if (p->d.L > 2048) return fail(SSHT_EUNSUPPORTED, "band-limit too large for the triangular solve");
  int rc = check_device(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = set_streams(p, st))) return rc;
  IO io;
  if ((rc = io_begin(p, f, p->grid_bytes(), flm, p->coeff_bytes(), st, &io))) return rc;
  const void* src = io.in_dev;
  void* dst = io.out_dev;
  if (p->real) {
    StageScope sc(p, SSHT_STAGE_PACK, st);
    SSHT_CUDA(real_pack_grid<double>(p->d.L, p->nreal, io.in_dev, p->rg, st), "real-field packing");
    p->launches += 1;
    src = p->rg;
    dst = p->rc;
  }
  if ((rc = begin_operands(p, 1, st))) return rc;
  if ((rc = analysis_front<double>(p, src, 0, st))) return rc;
  if ((rc = join_operands(p, st))) return rc;
  {
    StageScope sc(p, SSHT_STAGE_PROJECT, st);
    SSHT_CUDA(triangular_solve(p->d, p->s, p->B, p->delta.table, p->U, p->W1, p->ph64, dst, st), "triangular solve");
    p->launches += 2;
  }
  if ((rc = mark_free(p, st))) return rc;
  if (p->real) {
    StageScope sc(p, SSHT_STAGE_PACK, st);
    SSHT_CUDA(real_unpack_coeffs<double>(p->d.L, p->nreal, p->rc, io.out_dev, st), "real-field unpacking");
    p->launches += 1;
  }
  return io_end(p, io, st);
}

int ssht_wigner_delta(ssht_plan_t p, double* out, void* stream) {
  if (!p || !out) return fail(SSHT_EINVAL, "null argument");
  int rc = check_device(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = ensure_delta(p, st))) return rc;
  const size_t bytes = delta_offset(p->d.L) * sizeof(double);
  if (is_device_pointer(out)) {
    SSHT_CUDA(cudaMemcpyAsync(out, p->delta.table, bytes, cudaMemcpyDeviceToDevice, st), "Delta table copy");
  } else {
    SSHT_CUDA(cudaMemcpyAsync(out, p->delta.table, bytes, cudaMemcpyDeviceToHost, st), "Delta table copy");
    SSHT_CUDA(cudaStreamSynchronize(st), "stream synchronize");
  }
  if ((rc = mark_free(p, st))) return rc;  // the recursion above ran on st: later calls wait for it
  SSHT_CUDA(cudaGetLastError(), "kernel launch");
  return SSHT_OK;
}

int ssht_plan_check(ssht_plan_t p) {
  if (!p) return fail(SSHT_EINVAL, "null plan");
  int rc = check_device(p);
  if (rc) return rc;
  SSHT_CUDA(cudaDeviceSynchronize(), "device synchronize");
  int st = 0;
  SSHT_CUDA(cudaMemcpy(&st, p->delta.status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  if (st != 0) {
    cudaMemset(p->delta.status, 0, sizeof(int));
    if (p->delta_mode == SSHT_DELTA_CACHE) p->delta_ready = false;
    return fail(SSHT_ETIMEOUT, std::string("a device-side wait exceeded its spin limit (") +
                                   ((st & kStatusBarrierTimeout) ? "recursion hand-off" : "") +
                                   ((st & kStatusBarrierTimeout) && (st & 2) ? ", " : "") +
                                   ((st & 2) ? "tensor-core pipeline" : "") + ")");
  }
  return SSHT_OK;
}

int ssht_plan_tile_config(ssht_plan_t p, int* cfg) {
  if (!p || !cfg) return fail(SSHT_EINVAL, "null argument");
  if (!p->tc) return fail(SSHT_EUNSUPPORTED, "the plan has no tensor-core contraction");
  const TcConfig c = tc_config(p->tc);
  cfg[0] = c.slice;
  cfg[1] = c.stages;
  cfg[2] = c.inv_order;
  cfg[3] = c.fwd_order;
  return SSHT_OK;
}

int ssht_plan_set_wait_limit(ssht_plan_t p, long long ns) {
  if (!p) return fail(SSHT_EINVAL, "null plan");
  p->wait_ns = ns > 0 ? ns : kDefaultWaitNs;
  return SSHT_OK;
}

int ssht_plan_profile(ssht_plan_t p, int enable) {
  if (!p) return fail(SSHT_EINVAL, "null plan");
  int rc = check_device(p);
  if (rc) return rc;
  SSHT_CUDA(cudaDeviceSynchronize(), "device synchronize");
  for (auto& e : p->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  p->evs.clear();
  for (int i = 0; i < SSHT_NUM_STAGES; ++i) {
    p->prof_ms[i] = 0.0;
    p->prof_n[i] = 0;
  }
  p->prof = enable != 0;
  return SSHT_OK;
}

int ssht_plan_profile_read(ssht_plan_t p, double* ms, long long* count, int nstages, long long* launches) {
  if (!p) return fail(SSHT_EINVAL, "null plan");
  if (nstages < 0 || nstages > SSHT_NUM_STAGES || (nstages > 0 && (!ms || !count)))
    return fail(SSHT_EINVAL, "bad stage buffers");
  int rc = check_device(p);
  if (rc) return rc;
  SSHT_CUDA(cudaDeviceSynchronize(), "device synchronize");
  fold_events(p);
  for (int i = 0; i < nstages; ++i) {
    ms[i] = p->prof_ms[i];
    count[i] = p->prof_n[i];
  }
  if (launches) *launches = p->launches;
  return SSHT_OK;
}

int ssht_plan_profile_trace(ssht_plan_t p, int* stage, int* lane, double* t0, double* t1, int cap, int* n) {
  if (!p) return fail(SSHT_EINVAL, "null plan");
  if (!n || cap < 0 || (cap > 0 && (!stage || !lane || !t0 || !t1))) return fail(SSHT_EINVAL, "bad trace buffers");
  int rc = check_device(p);
  if (rc) return rc;
  SSHT_CUDA(cudaDeviceSynchronize(), "device synchronize");
  *n = (int)std::min(p->evs.size(), (size_t)cap);
  double first = 0.0;  // brackets of the two streams need not start in recording order
  for (int i = 0; i < *n; ++i) {
    const auto& e = p->evs[i];
    float a = 0.f, b = 0.f;
    SSHT_CUDA(cudaEventElapsedTime(&a, p->evs[0].a, e.a), "trace event time");
    SSHT_CUDA(cudaEventElapsedTime(&b, p->evs[0].a, e.b), "trace event time");
    stage[i] = e.stage;
    lane[i] = e.lane;
    t0[i] = a;
    t1[i] = b;
    first = std::min(first, (double)a);
  }
  for (int i = 0; i < *n; ++i) {
    t0[i] -= first;
    t1[i] -= first;
  }
  fold_events(p);
  return SSHT_OK;
}

const char* ssht_last_error(void) { return g_last_error.c_str(); }

int ssht_debug_fail_allocation(int n) {
  if (n < 0) return fail(SSHT_EINVAL, "ssht_debug_fail_allocation: n must be >= 0");
  g_alloc_countdown.store(n);
  return SSHT_OK;
}

int ssht_debug_bounds(long long* count, int* site, long long* index, long long* extent) {
  if (!kBoundsChecked) return fail(SSHT_EUNSUPPORTED, "ssht_debug_bounds: this library was built without index checks");
  SSHT_CUDA(cudaDeviceSynchronize(), "synchronize");
  cudaError_t (*take[])(BoundsRecord*) = {bounds_take_torus_pass, bounds_take_contract_tc, bounds_take_delta_column,
                                          bounds_take_real, bounds_take_contract_simt};
  BoundsRecord first{};
  long long total = 0;
  for (auto f : take) {
    BoundsRecord r{};
    SSHT_CUDA(f(&r), "index-check record");
    if (r.count && !total) first = r;
    total += (long long)r.count;
  }
  if (count) *count = total;
  if (site) *site = total ? first.kernel : 0;
  if (index) *index = total ? first.index : 0;
  if (extent) *extent = total ? first.extent : 0;
  return 0;
}

int ssht_version(void) { return 100; }

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Groups: many fields of uneven band-limit and spin in one call (and one CUDA graph).
//
// Fields are bucketed by (L, s); each bucket is one plan over its fields, which sit contiguously
// in the caller's flat buffers in group order (ssht_group_layout).  All buckets of one L share one
// Delta table: in recompute mode each call runs one recursion per distinct L, on its own stream,
// and the buckets wait for it before their spin column and packing; in cache mode the tables are
// made once here.  Buckets run on their own streams, forked from and joined to the caller's.
// With tuning on, each bucket times every contraction form of the group's precision class
// (FP32, 3xTF32, split-BF16 for FP32-class groups; the tensor-core forms with their own tuned
// shape) on its own shape and keeps the fastest.
// ---------------------------------------------------------------------------------------------

struct ssht_group_s {
  int device = 0;
  int n = 0;
  int precision = 0, delta_mode = 0;
  size_t elem = 8;
  std::vector<int> order;            // group position -> caller's field index
  std::vector<long long> coff, goff; // per group position: element offsets of coefficients / samples
  struct Holder {
    int L = 0;
    DeltaWork dw{};
    cudaEvent_t ev = nullptr;
  };
  // The shared recursions run one after another on one stream: each is a cooperative grid over
  // every SM, so running two at once would only make them wait for each other's SMs.
  cudaStream_t rec_st = nullptr;
  std::vector<Holder> holders;
  struct Bucket {
    int L = 0, s = 0, first = 0, count = 0, holder = 0;
    ssht_plan_t plan = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
  };
  std::vector<Bucket> buckets;
  cudaEvent_t ev_start = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void group_release(ssht_group_t g) {
  if (!g) return;
  cudaDeviceSynchronize();
  if (g->exec) cudaGraphExecDestroy(g->exec);
  for (auto& b : g->buckets) {
    if (b.plan) release(b.plan);
    if (b.st) cudaStreamDestroy(b.st);
    if (b.ev) cudaEventDestroy(b.ev);
  }
  for (auto& h : g->holders) {
    delta_free(h.dw);
    if (h.ev) cudaEventDestroy(h.ev);
  }
  if (g->rec_st) cudaStreamDestroy(g->rec_st);
  if (g->ev_start) cudaEventDestroy(g->ev_start);
  delete g;
}

// One call of every bucket; which: 0 inverse, 1 forward, 2 adjoint.
int group_call(ssht_group_t g, int which, const void* in, void* out, cudaStream_t st) {
  SSHT_CUDA(cudaEventRecord(g->ev_start, st), "group fork");
  if (g->delta_mode == SSHT_DELTA_RECOMPUTE) {
    SSHT_CUDA(cudaStreamWaitEvent(g->rec_st, g->ev_start, 0), "group fork wait");
    for (auto& h : g->holders) {
      SSHT_CUDA(delta_run(h.dw, h.L, g->rec_st), "shared Delta recursion");
      SSHT_CUDA(cudaEventRecord(h.ev, g->rec_st), "shared Delta event");
    }
  }
  for (auto& b : g->buckets) {
    ssht_plan_t p = b.plan;
    SSHT_CUDA(cudaStreamWaitEvent(b.st, g->ev_start, 0), "group fork wait");
    p->delta_event = g->delta_mode == SSHT_DELTA_RECOMPUTE ? g->holders[b.holder].ev : nullptr;
    int rc = set_streams(p, b.st);
    if (rc) return rc;
    const long long ci = g->coff[b.first], gi = g->goff[b.first];
    const char* src = (const char*)in + (which == 0 ? ci : gi) * g->elem;
    char* dst = (char*)out + (which == 0 ? gi : ci) * g->elem;
    if (which == 0)
      rc = p->f64 ? inverse_impl<double>(p, src, dst, b.st) : inverse_impl<float>(p, src, dst, b.st);
    else if (which == 1)
      rc = p->f64 ? forward_impl<double>(p, src, dst, b.st) : forward_impl<float>(p, src, dst, b.st);
    else
      rc = p->f64 ? adjoint_impl<double>(p, src, dst, b.st) : adjoint_impl<float>(p, src, dst, b.st);
    if (rc) return rc;
    SSHT_CUDA(cudaEventRecord(b.ev, b.st), "group join event");
  }
  for (auto& b : g->buckets) SSHT_CUDA(cudaStreamWaitEvent(st, b.ev, 0), "group join wait");
  return 0;
}

// Mean milliseconds of inverse + forward of one plan on zero data (shapes decide the time).
int time_plan(ssht_plan_t p, float* ms) {
  void *a = nullptr, *b = nullptr, *c = nullptr;
  const size_t cb = p->coeff_bytes(), gb = p->grid_bytes();
  int rc = 0;
  if ((rc = dalloc(p, &a, cb, "tuning input")) || (rc = dalloc(p, &b, gb, "tuning grid")) ||
      (rc = dalloc(p, &c, cb, "tuning output"))) {
    cudaFree(a);
    cudaFree(b);
    return rc;
  }
  p->bytes -= cb + gb + cb;
  cudaEvent_t e0, e1;
  cudaStream_t st = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaMemsetAsync(a, 0, cb, st);
  for (int it = 0; it < 6 && !rc; ++it) {
    if (it == 2) cudaEventRecord(e0, st);
    rc = p->f64 ? inverse_impl<double>(p, a, b, st) : inverse_impl<float>(p, a, b, st);
    if (!rc) rc = p->f64 ? forward_impl<double>(p, b, c, st) : forward_impl<float>(p, b, c, st);
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  *ms = t / 4.f;
  cudaStreamDestroy(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(a);
  cudaFree(b);
  cudaFree(c);
  return rc;
}

int group_create(ssht_group_t* out, int n, const int* Ls, const int* ss, int precision, int delta_mode, int tune) {
  if (!out || !Ls || !ss) return fail(SSHT_EINVAL, "null argument");
  *out = nullptr;
  if (n < 1) return fail(SSHT_EINVAL, "a group needs at least one field");
  if (precision != SSHT_FP64 && precision != SSHT_FP32 && precision != SSHT_TF32X3 && precision != SSHT_BF16X6)
    return fail(SSHT_EINVAL, "unknown precision");
  if (delta_mode != SSHT_DELTA_RECOMPUTE && delta_mode != SSHT_DELTA_CACHE) return fail(SSHT_EINVAL, "unknown Delta mode");
  for (int i = 0; i < n; ++i) {
    if (Ls[i] < 1 || Ls[i] > 2048) return fail(SSHT_EINVAL, "band-limit L must be in [1, 2048]");
    if (ss[i] <= -Ls[i] || ss[i] >= Ls[i]) return fail(SSHT_EINVAL, "spin must satisfy |s| < L");
  }
  ssht_group_t g = new (std::nothrow) ssht_group_s();
  if (!g) return fail(SSHT_ENOMEM, "host allocation of the group");
  auto bail = [&](int code) {
    group_release(g);
    return code;
  };
  cudaError_t ce = cudaGetDevice(&g->device);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&g->ev_start, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&g->rec_st, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return bail(fail(SSHT_ECUDA, std::string("group setup: ") + cudaGetErrorString(ce)));
  g->n = n;
  g->precision = precision;
  g->delta_mode = delta_mode;
  g->elem = precision == SSHT_FP64 ? 16 : 8;
  // group order: by L, then s, then the caller's index
  g->order.resize(n);
  for (int i = 0; i < n; ++i) g->order[i] = i;
  std::stable_sort(g->order.begin(), g->order.end(),
                   [&](int a, int b) { return Ls[a] != Ls[b] ? Ls[a] < Ls[b] : ss[a] < ss[b]; });
  g->coff.resize(n + 1);
  g->goff.resize(n + 1);
  long long c = 0, q = 0;
  for (int k = 0; k < n; ++k) {
    const int L = Ls[g->order[k]];
    g->coff[k] = c;
    g->goff[k] = q;
    c += (long long)L * L;
    q += (long long)L * (2 * L - 1);
  }
  g->coff[n] = c;
  g->goff[n] = q;
  // shared Delta tables, one per distinct L
  for (int k = 0; k < n; ++k) {
    const int L = Ls[g->order[k]];
    if (g->holders.empty() || g->holders.back().L != L) {
      g->holders.emplace_back();
      auto& h = g->holders.back();
      h.L = L;
      ce = delta_setup(h.dw, L, g->device);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h.ev, cudaEventDisableTiming);
      if (ce == cudaSuccess) ce = delta_run(h.dw, L, 0);  // valid tables for tuning and cache mode
      if (ce != cudaSuccess)
        return bail(fail(ce == cudaErrorMemoryAllocation ? SSHT_ENOMEM : SSHT_ECUDA,
                         std::string("shared Delta setup: ") + cudaGetErrorString(ce)));
    }
  }
  ce = cudaDeviceSynchronize();
  if (ce != cudaSuccess) return bail(fail(SSHT_ECUDA, std::string("shared Delta: ") + cudaGetErrorString(ce)));
  // buckets
  for (int k = 0; k < n;) {
    const int L = Ls[g->order[k]], s = ss[g->order[k]];
    int e = k;
    while (e < n && Ls[g->order[e]] == L && ss[g->order[e]] == s) ++e;
    g->buckets.emplace_back();
    auto& b = g->buckets.back();
    b.L = L;
    b.s = s;
    b.first = k;
    b.count = e - k;
    b.holder = (int)g->holders.size() - 1;
    while (g->holders[b.holder].L != L) --b.holder;
    ce = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(fail(SSHT_ECUDA, "bucket stream setup"));
    std::vector<int> cands;
    if (!tune || precision == SSHT_FP64) {
      cands.push_back(precision);
    } else {
      cands.push_back(SSHT_FP32);
      cands.push_back(SSHT_TF32X3);
      cands.push_back(SSHT_BF16X6);
    }
    float best = 0.f;
    for (int cand : cands) {
      ssht_plan_desc d{L, s, b.count, cand, delta_mode,
                       (tune && (cand == SSHT_TF32X3 || cand == SSHT_BF16X6)) ? SSHT_FLAG_TUNE : 0};
      ssht_plan_t p = nullptr;
      int rc = create(&p, &d, &g->holders[b.holder].dw);
      if (rc) return bail(rc);
      float ms = 0.f;
      if (cands.size() > 1 && (rc = time_plan(p, &ms))) {
        release(p);
        return bail(rc);
      }
      if (!b.plan || ms < best) {
        if (b.plan) release(b.plan);
        b.plan = p;
        best = ms;
      } else {
        release(p);
      }
    }
    k = e;
  }
  *out = g;
  g_last_error.clear();
  return SSHT_OK;
}

}  // namespace

extern "C" {

int ssht_group_create(ssht_group_t* out, int n, const int* L, const int* s, int precision, int delta_mode, int tune) {
  return group_create(out, n, L, s, precision, delta_mode, tune);
}

int ssht_group_destroy(ssht_group_t g) {
  group_release(g);
  return SSHT_OK;
}

int ssht_group_layout(ssht_group_t g, int* order, long long* coeff_offset, long long* grid_offset) {
  if (!g) return fail(SSHT_EINVAL, "null group");
  for (int k = 0; k < g->n; ++k) {
    if (order) order[k] = g->order[k];
    if (coeff_offset) coeff_offset[k] = g->coff[k];
    if (grid_offset) grid_offset[k] = g->goff[k];
  }
  if (coeff_offset) coeff_offset[g->n] = g->coff[g->n];
  if (grid_offset) grid_offset[g->n] = g->goff[g->n];
  return SSHT_OK;
}

int ssht_group_buckets(ssht_group_t g, int* nbuckets, int* L, int* s, int* count, int* precision) {
  if (!g || !nbuckets) return fail(SSHT_EINVAL, "null argument");
  const int nb = (int)g->buckets.size();
  const int cap = *nbuckets;
  *nbuckets = nb;
  for (int i = 0; i < nb && i < cap; ++i) {
    if (L) L[i] = g->buckets[i].L;
    if (s) s[i] = g->buckets[i].s;
    if (count) count[i] = g->buckets[i].count;
    if (precision) precision[i] = g->buckets[i].plan->precision;
  }
  return SSHT_OK;
}

int ssht_group_bucket_tile_config(ssht_group_t g, int bucket, int* cfg) {
  if (!g || !cfg) return fail(SSHT_EINVAL, "null argument");
  if (bucket < 0 || bucket >= (int)g->buckets.size()) return fail(SSHT_EINVAL, "no such bucket");
  return ssht_plan_tile_config(g->buckets[bucket].plan, cfg);
}

static int group_entry(ssht_group_t g, int which, const void* in, void* out, void* stream) {
  if (!g || !in || !out) return fail(SSHT_EINVAL, "null argument");
  int cur = -1;
  SSHT_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
  if (cur != g->device) return fail(SSHT_EINVAL, "group used on another device");
  if (!is_device_pointer(in) || !is_device_pointer(out)) return fail(SSHT_EINVAL, "group buffers must be device memory");
  return group_call(g, which, in, out, (cudaStream_t)stream);
}

int ssht_group_inverse(ssht_group_t g, const void* flm, void* f, void* stream) { return group_entry(g, 0, flm, f, stream); }
int ssht_group_forward(ssht_group_t g, const void* f, void* flm, void* stream) { return group_entry(g, 1, f, flm, stream); }
int ssht_group_adjoint(ssht_group_t g, const void* f, void* flm, void* stream) { return group_entry(g, 2, f, flm, stream); }

int ssht_group_capture(ssht_group_t g, const void* flm, void* f, void* flm_out, void* stream) {
  if (!g || !flm || !f || !flm_out) return fail(SSHT_EINVAL, "null argument");
  if (!is_device_pointer(flm) || !is_device_pointer(f) || !is_device_pointer(flm_out))
    return fail(SSHT_EINVAL, "group buffers must be device memory");
  (void)stream;  // capturing launches nothing: it records on a private stream (the legacy default
                 // stream cannot be captured)
  cudaStream_t cap = nullptr;
  SSHT_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
  if (g->exec) {
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int rc = 0;
  if (ce == cudaSuccess) {
    rc = group_call(g, 0, flm, f, cap);
    if (!rc) rc = group_call(g, 1, f, flm_out, cap);
    ce = cudaStreamEndCapture(cap, &graph);
  }
  if (ce == cudaSuccess && !rc) ce = cudaGraphInstantiate(&g->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (rc) return rc;
  if (ce != cudaSuccess) return fail(SSHT_ECUDA, std::string("group graph capture: ") + cudaGetErrorString(ce));
  return SSHT_OK;
}

int ssht_group_replay(ssht_group_t g, void* stream) {
  if (!g || !g->exec) return fail(SSHT_EINVAL, "no captured graph");
  SSHT_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream), "graph launch");
  return SSHT_OK;
}

int ssht_group_check(ssht_group_t g) {
  if (!g) return fail(SSHT_EINVAL, "null group");
  SSHT_CUDA(cudaDeviceSynchronize(), "device synchronize");
  for (auto& h : g->holders) {
    int st = 0;
    SSHT_CUDA(cudaMemcpy(&st, h.dw.status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
    if (st != 0) {
      cudaMemset(h.dw.status, 0, sizeof(int));
      return fail(SSHT_ETIMEOUT, "a Delta recursion wait exceeded its spin limit");
    }
  }
  return SSHT_OK;
}

}  // extern "C"
