// Krylov solver (S10): left-preconditioned restarted GMRES with classical
// Gram-Schmidt applied twice (CGS2), inner products accumulated in FP64 on the
// device (Sect. 5.1-5.2).  The Arnoldi coefficients never leave the device:
// the Gram-Schmidt projections read them from device memory, and one
// single-thread kernel per iteration applies the Givens rotations to the new
// Hessenberg column, forms the next rotation and the residual estimate (FP64).
// The host reads back that estimate once per iteration (to stop), and the
// least-squares back substitution runs on the device at the end of a cycle.
// The step index j lives in device memory too, so one Arnoldi step (operator,
// preconditioner, both Gram-Schmidt passes, the rotation kernel, the scaled
// next basis vector and the copy of the scalars to pinned host memory) is the
// same launch sequence for every j: it is captured once per context as a CUDA
// graph and replayed, one graph launch per iteration.
// The stopping test is the unpreconditioned relative residual ||b - A x|| /
// ||b|| of Sect. 5.1, recomputed in FP64 before returning.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <map>
#include <vector>
#include "prd_internal.h"
#include "device_common.cuh"
#include "lockstep.h"

namespace prd {

// dots[k] += sum_i V[k][i] * w[i]   for k < nv   (FP64 accumulation)
template <typename T>
__global__ void multidot_kernel(const T* __restrict__ V, size_t ld, const T* __restrict__ w, size_t n, double* dots) {
  const int k = blockIdx.y;
  const T* v = V + (size_t)k * ld;
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += (double)v[i] * (double)w[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&dots[k], red[0]);
}

// x += sum_k y[k] V[k]   (y in device memory)
template <typename T>
__global__ void update_kernel(const T* __restrict__ V, size_t ld, const double* __restrict__ y, int nv, T* x, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = (double)x[i];
    for (int k = 0; k < nv; ++k) s += y[k] * (double)V[(size_t)k * ld + i];
    x[i] = (T)s;
  }
}

// r = b - r   (r holds A x on entry)
template <typename T>
__global__ void rsub_kernel(const T* __restrict__ b, T* r, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    r[i] = b[i] - r[i];
}

// Device state of one GMRES(m) cycle, in one FP64 array:
//   H[(m+1) x m] (row-major, the rotated Hessenberg matrix), cs[m], sn[m],
//   g[m+1] (rotated right-hand side), y[m] (least-squares solution),
//   h[m+1], h2[m+1] (projections of the two Gram-Schmidt passes), and
//   scalars: kSS (sum of squares), kInv (1/norm for scaling), kEst (residual
//   estimate), kNorm (norm), kBeta0.
struct GState {
  int m;
  __host__ __device__ size_t H() const { return 0; }
  __host__ __device__ size_t cs() const { return (size_t)(m + 1) * m; }
  __host__ __device__ size_t sn() const { return cs() + m; }
  __host__ __device__ size_t g() const { return sn() + m; }
  __host__ __device__ size_t y() const { return g() + m + 1; }
  __host__ __device__ size_t h() const { return y() + m; }
  __host__ __device__ size_t h2() const { return h() + m + 1; }
  __host__ __device__ size_t sc() const { return h2() + m + 1; }
  __host__ __device__ size_t total() const { return sc() + 8; }
};
enum { kSS = 0, kInv = 1, kEst = 2, kNorm = 3, kBeta0 = 4, kJ = 5, kTr = 6 };

// dots[k] = sum_i V[k][i] * w[i] for k <= j, j = st[kJ] read on the device
// (dots zeroed by the caller); blocks stride over k so the grid is fixed
template <typename T>
__global__ void multidot_j_kernel(const T* __restrict__ V, size_t ld, const T* __restrict__ w, size_t n,
                                  const double* __restrict__ sc, double* dots) {
  const int nv = (int)sc[kJ] + 1;
  __shared__ double red[256];
  for (int k = blockIdx.y; k < nv; k += gridDim.y) {
    const T* v = V + (size_t)k * ld;
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
      s += (double)v[i] * (double)w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
      if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&dots[k], red[0]);
    __syncthreads();
  }
}

// w -= sum_{k <= j} h[k] V[k],  j = st[kJ]
template <typename T>
__global__ void multiaxpy_j_kernel(const T* __restrict__ V, size_t ld, const double* __restrict__ h,
                                   const double* __restrict__ sc, T* w, size_t n) {
  const int nv = (int)sc[kJ] + 1;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = (double)w[i];
    for (int k = 0; k < nv; ++k) s -= h[k] * (double)V[(size_t)k * ld + i];
    w[i] = (T)s;
  }
}

// V[j] = cur = a * st[kInv],  j = st[kJ] (the basis vector the next step applies A to)
template <typename T>
__global__ void scale_j_kernel(const T* __restrict__ a, const double* __restrict__ sc, T* __restrict__ V, size_t ld,
                               T* __restrict__ cur, size_t n) {
  const double f = sc[kInv];
  T* dst = V + (size_t)(int)sc[kJ] * ld;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T v = (T)((double)a[i] * f);
    dst[i] = v;
    cur[i] = v;
  }
}

// start of a cycle: beta = sqrt(ss); g = beta e_1; 1/beta for the first basis vector
__global__ void gm_cycle_start_kernel(double* st, GState L, double tr) {
  double* sc = st + L.sc();
  const double beta = sqrt(sc[kSS]);
  double* g = st + L.g();
  for (int i = 0; i <= L.m; ++i) g[i] = 0.0;
  g[0] = beta;
  sc[kBeta0] = beta;
  sc[kNorm] = beta;
  sc[kInv] = beta > 0.0 ? 1.0 / beta : 0.0;
  sc[kJ] = 0.0;
  sc[kTr] = tr;
}

// Arnoldi step j: Hessenberg column from the two Gram-Schmidt passes and the
// norm of the orthogonalised vector, earlier rotations applied, the new
// rotation formed and applied to g; estimate tr |g[j+1]| / beta0.
__global__ void gm_arnoldi_kernel(double* st, GState L) {
  const int m = L.m;
  const int j = (int)st[L.sc() + kJ];
  const double tr = st[L.sc() + kTr];
  double* H = st + L.H();
  double* cs = st + L.cs();
  double* sn = st + L.sn();
  double* g = st + L.g();
  const double* h = st + L.h();
  const double* h2 = st + L.h2();
  double* sc = st + L.sc();
  const double hn = sqrt(sc[kSS]);
  for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i] + h2[i];
  H[(size_t)(j + 1) * m + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a0 = H[(size_t)i * m + j], a1 = H[(size_t)(i + 1) * m + j];
    H[(size_t)i * m + j] = cs[i] * a0 + sn[i] * a1;
    H[(size_t)(i + 1) * m + j] = -sn[i] * a0 + cs[i] * a1;
  }
  const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
  const double den = hypot(a0, a1);
  cs[j] = den > 0 ? a0 / den : 1.0;
  sn[j] = den > 0 ? a1 / den : 0.0;
  H[(size_t)j * m + j] = den;
  H[(size_t)(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  sc[kNorm] = hn;
  sc[kInv] = hn > 0.0 ? 1.0 / hn : 0.0;
  sc[kEst] = tr * fabs(g[j + 1]) / sc[kBeta0];
  sc[kJ] = (double)(j + 1);
}

// y = H(0:j, 0:j)^-1 g(0:j)  (upper triangular after the rotations)
__global__ void gm_backsolve_kernel(double* st, GState L, int j) {
  const int m = L.m;
  const double* H = st + L.H();
  const double* g = st + L.g();
  double* y = st + L.y();
  for (int i = j - 1; i >= 0; --i) {
    double s = g[i];
    for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
    const double d = H[(size_t)i * m + i];
    y[i] = d != 0.0 ? s / d : 0.0;   // an exact breakdown on the first step leaves a zero pivot
  }
}

namespace {

struct Vops {
  Ctx* c;
  size_t n;
  int grid = 0;
  int init() {
    grid = c->grid_ew();
    return PRD_OK;
  }
  // out[k] = <V[k], w> for k < nv, in device memory
  int dot_many(const void* V, size_t ld, int nv, const void* w, double* out) {
    PRD_CUDA_TRY(c, cudaMemsetAsync(out, 0, nv * sizeof(double), c->stream));
    if (c->prec == PRD_FP64)
      multidot_kernel<double><<<dim3(grid, nv), 256, 0, c->stream>>>((const double*)V, ld, (const double*)w, n, out);
    else
      multidot_kernel<float><<<dim3(grid, nv), 256, 0, c->stream>>>((const float*)V, ld, (const float*)w, n, out);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
    return PRD_OK;
  }
  int update(const void* V, size_t ld, const double* y, int nv, void* x) {
    if (c->prec == PRD_FP64)
      update_kernel<double><<<grid, 256, 0, c->stream>>>((const double*)V, ld, y, nv, (double*)x, n);
    else
      update_kernel<float><<<grid, 256, 0, c->stream>>>((const float*)V, ld, y, nv, (float*)x, n);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
    return PRD_OK;
  }
  int rsub(const void* b, void* r) {
    if (c->prec == PRD_FP64) rsub_kernel<double><<<grid, 256, 0, c->stream>>>((const double*)b, (double*)r, n);
    else rsub_kernel<float><<<grid, 256, 0, c->stream>>>((const float*)b, (float*)r, n);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
    return PRD_OK;
  }
  // dots[k] = <V[k], w> for k <= j (device j), dots zeroed first
  int dot_j(const void* V, size_t ld, const void* w, const double* sc, double* dots, int m) {
    PRD_CUDA_TRY(c, cudaMemsetAsync(dots, 0, (m + 1) * sizeof(double), c->stream));
    const dim3 g(grid, 8);
    if (c->prec == PRD_FP64)
      multidot_j_kernel<double><<<g, 256, 0, c->stream>>>((const double*)V, ld, (const double*)w, n, sc, dots);
    else
      multidot_j_kernel<float><<<g, 256, 0, c->stream>>>((const float*)V, ld, (const float*)w, n, sc, dots);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
    return PRD_OK;
  }
  int axpy_j(const void* V, size_t ld, const double* h, const double* sc, void* w) {
    if (c->prec == PRD_FP64)
      multiaxpy_j_kernel<double><<<grid, 256, 0, c->stream>>>((const double*)V, ld, h, sc, (double*)w, n);
    else
      multiaxpy_j_kernel<float><<<grid, 256, 0, c->stream>>>((const float*)V, ld, h, sc, (float*)w, n);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
    return PRD_OK;
  }
  int scale_j(const void* a, const double* sc, void* V, void* cur) {
    if (c->prec == PRD_FP64)
      scale_j_kernel<double><<<grid, 256, 0, c->stream>>>((const double*)a, sc, (double*)V, n, (double*)cur, n);
    else
      scale_j_kernel<float><<<grid, 256, 0, c->stream>>>((const float*)a, sc, (float*)V, n, (float*)cur, n);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
    return PRD_OK;
  }
  // copy `cnt` doubles of device state to the host (synchronises the stream)
  int read(const double* src, double* dst, int cnt) {
    PRD_CUDA_TRY(c, cudaMemcpyAsync(dst, src, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PRD_OK;
  }
  // ||a|| on the host (sum of squares into *ss on the device)
  int norm(const void* a, double* ss, double* out) {
    int rc = dot_many(a, 0, 1, a, ss);
    if (rc) return rc;
    double h;
    if ((rc = read(ss, &h, 1))) return rc;
    *out = std::sqrt(h);
    return PRD_OK;
  }
};

}  // namespace

int apply_operator_t(Ctx* c, const void* x, void* y);
// the operator GMRES iterates with: A, or A^T for the adjoint solve (or the
// zero map injected for testing the breakdown path, PRD_OPT_TEST_ZERO_OPERATOR)
static int op_apply(Ctx* c, const void* x, void* y) {
  if (c->test_zero_op) {
    PRD_CUDA_TRY(c, cudaMemsetAsync(y, 0, nvec(c) * c->esz, c->stream));
    return PRD_OK;
  }
  return c->op_transpose ? apply_operator_t(c, x, y) : apply_operator(c, x, y);
}

void invalidate_graphs(Ctx* c) {
  for (auto& g : c->gk_exec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (auto& g : c->gk_graph)
    if (g) {
      cudaGraphDestroy(g);
      g = nullptr;
    }
}

// ---- lockstep rounds of prd_solve_batch (the round logic: lockstep.h)
using BatchReq = std::pair<Ctx*, int>;       // (context, graph key) waiting in a round
struct BatchRound {
  explicit BatchRound(int n) : ls(n) {}
  Lockstep<BatchReq> ls;
  cudaStream_t stream = nullptr;             // the rounds' launch stream
  cudaEvent_t ev = nullptr;
  std::map<std::vector<BatchReq>, cudaGraphExec_t> cache;   // by the set of children
  long long launches = 0;
};

BatchRound* batch_round_create(int n) {
  BatchRound* b = new BatchRound(n);
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
    batch_round_destroy(b);
    return nullptr;
  }
  return b;
}

void batch_round_destroy(BatchRound* b) {
  if (!b) return;
  for (auto& kv : b->cache) cudaGraphExecDestroy(kv.second);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Launch the round for the waiting contexts (run under the round's lock): the
// launch stream waits for each context's stream, one launch of the graph with
// their steps as children, then the host waits for it.
static int batch_round_launch(BatchRound* b, const std::vector<BatchReq>& req) {
  std::vector<BatchReq> key = req;
  std::sort(key.begin(), key.end());
  cudaError_t e = cudaSuccess;
  auto it = b->cache.find(key);
  if (it == b->cache.end()) {
    cudaGraph_t pg = nullptr;
    e = cudaGraphCreate(&pg, 0);
    for (size_t i = 0; e == cudaSuccess && i < key.size(); ++i) {
      cudaGraphNode_t node;
      e = cudaGraphAddChildGraphNode(&node, pg, nullptr, 0, key[i].first->gk_graph[key[i].second]);
    }
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, pg, 0);
    if (pg) cudaGraphDestroy(pg);
    if (e != cudaSuccess) return (int)e;
    it = b->cache.emplace(key, ex).first;
  }
  for (auto& r : key) {
    if (e == cudaSuccess) e = cudaEventRecord(b->ev, r.first->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev, 0);
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(it->second, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) {
    ++b->launches;
    for (auto& r : key) ++r.first->gk_launches;
  }
  return (int)e;
}

// A context's Arnoldi step inside a batch round: wait for the round (the last
// context to arrive launches it) and return its status.
static cudaError_t batch_round_step(BatchRound* b, Ctx* c, int key) {
  return (cudaError_t)b->ls.arrive(BatchReq(c, key),
                                   [b](const std::vector<BatchReq>& req) { return batch_round_launch(b, req); });
}

// A context stops taking part (its solve ended, or it runs its steps one by
// one from now on); if everyone left is waiting, their round is launched.
void batch_round_leave(BatchRound* b) {
  if (!b) return;
  b->ls.leave([b](const std::vector<BatchReq>& req) { return batch_round_launch(b, req); });
}

// GMRES workspace of restart length m, kept by the context (the captured step
// refers to its addresses); reallocated, and the graphs dropped, when m grows.
static int gmres_workspace(Ctx* c, int m) {
  if (c->gk_m >= m && c->gk_V.p) return PRD_OK;
  invalidate_graphs(c);
  dfree(c->gk_V); dfree(c->gk_r); dfree(c->gk_w); dfree(c->gk_cur); dfree(c->gk_S);
  c->gk_m = 0;
  const size_t vb = nvec(c) * c->esz;
  const GState L{m};
  int rc;
  if ((rc = dalloc(c, c->gk_V, vb * (m + 1))) || (rc = dalloc(c, c->gk_r, vb)) || (rc = dalloc(c, c->gk_w, vb)) ||
      (rc = dalloc(c, c->gk_cur, vb)) || (rc = dalloc(c, c->gk_S, L.total() * sizeof(double))))
    return rc;
  if (!c->gk_host) PRD_CUDA_TRY(c, cudaMallocHost((void**)&c->gk_host, 8 * sizeof(double)));
  c->gk_m = m;
  return PRD_OK;
}

// One Arnoldi step on the context's workspace (restart length L.m): w = A cur,
// r = P^-1 w, two Gram-Schmidt passes against V[0..j], ||r||^2, the rotation
// kernel (j -> j + 1), V[j + 1] = cur = r / ||r||, and the scalars copied to
// pinned host memory.  Every address and launch shape is independent of j.
static int record_step(Ctx* c, Vops& ops, const GState& L) {
  const size_t n = nvec(c);
  double* st = (double*)c->gk_S.p;
  const double* sc = st + L.sc();
  int rc;
  if ((rc = op_apply(c, c->gk_cur.p, c->gk_w.p)) || (rc = apply_precond(c, c->gk_w.p, c->gk_r.p)) ||
      (rc = ops.dot_j(c->gk_V.p, n, c->gk_r.p, sc, st + L.h(), L.m)) ||
      (rc = ops.axpy_j(c->gk_V.p, n, st + L.h(), sc, c->gk_r.p)) ||
      (rc = ops.dot_j(c->gk_V.p, n, c->gk_r.p, sc, st + L.h2(), L.m)) ||
      (rc = ops.axpy_j(c->gk_V.p, n, st + L.h2(), sc, c->gk_r.p)) ||
      (rc = ops.dot_many(c->gk_r.p, 0, 1, c->gk_r.p, st + L.sc() + kSS)))
    return rc;
  gm_arnoldi_kernel<<<1, 1, 0, c->stream>>>(st, L);
  if ((rc = ops.scale_j(c->gk_r.p, sc, c->gk_V.p, c->gk_cur.p))) return rc;
  PRD_CUDA_TRY(c, cudaMemcpyAsync(c->gk_host, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return PRD_OK;
}

// Run one Arnoldi step and wait for its scalars: replay the captured graph
// (captured on first use), or launch directly (graphs off, or stage profiling
// on, whose events are host-timed per launch).
static int arnoldi_step(Ctx* c, Vops& ops, const GState& L, double* sc_host) {
  const int key = c->op_transpose ? 1 : 0;
  int rc = PRD_OK;
  if (c->use_graph && !c->prof && !c->test_zero_op && !c->gk_exec[key]) {
    // capture on the context's private stream (the caller's may be the legacy
    // default stream, which cannot be captured); the graph is launched on the
    // caller's.  A step that cannot be captured runs as direct launches from then on.
    bool ok = c->gk_cap || cudaStreamCreateWithFlags(&c->gk_cap, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(c->stream) == cudaSuccess;
    cudaStream_t user = c->stream;
    if (ok) ok = cudaStreamBeginCapture(c->gk_cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      c->stream = c->gk_cap;
      rc = record_step(c, ops, L);
      c->stream = user;
      cudaGraph_t g = nullptr;
      ok = cudaStreamEndCapture(c->gk_cap, &g) == cudaSuccess && rc == PRD_OK && g &&
           cudaGraphInstantiate(&c->gk_exec[key], g, 0) == cudaSuccess;
      if (ok) c->gk_graph[key] = g;
      else if (g) cudaGraphDestroy(g);
    }
    if (!ok) {
      invalidate_graphs(c);
      c->use_graph = 0;
      cudaGetLastError();
      c->err = "ok";
    }
  }
  const bool graph = c->use_graph && !c->prof && !c->test_zero_op && c->gk_exec[key];
  if (c->batch && !graph) {
    // this context runs its steps one by one: it no longer holds up the rounds
    batch_round_leave(c->batch);
    c->batch = nullptr;
  }
  if (c->batch) {
    const cudaError_t e = batch_round_step(c->batch, c, key);
    if (e != cudaSuccess) return fail(c, PRD_E_CUDA, std::string("batched Arnoldi round: ") + cudaGetErrorString(e));
    std::memcpy(sc_host, c->gk_host, 8 * sizeof(double));
    return PRD_OK;
  }
  if (graph) {
    PRD_CUDA_TRY(c, cudaGraphLaunch(c->gk_exec[key], c->stream));
    ++c->gk_launches;
  } else if ((rc = record_step(c, ops, L))) {
    return rc;
  }
  PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::memcpy(sc_host, c->gk_host, 8 * sizeof(double));
  return PRD_OK;
}

// GMRES on A x = b in the ctx precision; x holds the initial guess on entry.
// inner: correction solve of the mixed-precision refinement.  x is zero on
// entry and the solve ends as soon as the Arnoldi estimate is below tol (the
// refinement's FP64 residual is the true check), so no apply is spent on a
// residual the caller recomputes anyway.
static int gmres_core(Ctx* c, const void* bvec, void* x, double tol, int max_iter, int restart, int* iters,
                      double* true_res, double* hist, double hist_scale, int* nh_io, bool inner = false) {
  const size_t n = nvec(c);
  const size_t vb = n * c->esz;
  const int m = std::max(1, std::min(restart, 200));
  Vops ops{c, n};
  int rc = ops.init();
  if (rc) return rc;
  if ((rc = gmres_workspace(c, m))) return rc;
  const GState L{c->gk_m};                  // the workspace's layout (restart length >= m)
  void* r = c->gk_r.p;
  void* w = c->gk_w.p;
  struct { void* p; } b{const_cast<void*>(bvec)};
  double* st = (double*)c->gk_S.p;
  double* ss = st + L.sc() + kSS;
  double bnorm;
  if ((rc = ops.norm(b.p, ss, &bnorm))) return rc;
  if (!(bnorm > 0) || !std::isfinite(bnorm)) return fail(c, PRD_E_NAN, "right-hand side norm is zero or not finite");
  int it = 0, nh = nh_io ? *nh_io : 0;
  double tol_in = tol;
  double tr = 1.0;
  int status = PRD_E_NOCONV;
  bool first = true;
  double sc[8];
  while (it < max_iter) {
    // r = P^-1 (b - A x)
    if (inner && first) {
      PRD_CUDA_TRY(c, cudaMemcpyAsync(w, b.p, vb, cudaMemcpyDeviceToDevice, c->stream));
      tr = 1.0;
    } else {
      if ((rc = op_apply(c, x, w)) || (rc = ops.rsub(b.p, w))) break;
      double rn_true;
      if ((rc = ops.norm(w, ss, &rn_true))) break;
      tr = rn_true / bnorm;
    }
    first = false;
    if (!std::isfinite(tr)) { rc = fail(c, PRD_E_NAN, "residual is not finite"); break; }
    if (tr < tol) { status = PRD_OK; break; }
    if ((rc = apply_precond(c, w, r))) break;
    if ((rc = ops.dot_many(r, 0, 1, r, ss))) break;
    gm_cycle_start_kernel<<<1, 1, 0, c->stream>>>(st, L, tr);
    // V[0] = cur = r / beta
    if ((rc = ops.scale_j(r, st + L.sc(), c->gk_V.p, c->gk_cur.p))) break;
    if ((rc = ops.read(st + L.sc(), sc, 8))) break;
    const double beta0 = sc[kBeta0];
    if (!(beta0 > 0)) { status = PRD_OK; break; }
    int j = 0;
    bool breakdown = false, est_ok = false;
    for (; j < m && it < max_iter; ++j) {
      if ((rc = arnoldi_step(c, ops, L, sc))) break;
      ++it;
      const double hn = sc[kNorm], est = sc[kEst];
      if (!std::isfinite(hn) || !std::isfinite(est)) { rc = fail(c, PRD_E_NAN, "Arnoldi vector is not finite"); break; }
      if (hist && nh <= max_iter) hist[nh++] = est * hist_scale;
      if (hn <= 1e-300 * std::max(1.0, beta0)) { breakdown = true; ++j; break; }
      if (est < 0.5 * tol_in) { ++j; est_ok = true; break; }
    }
    if (rc) break;
    // back substitution H y = g and x += V y, on the device
    gm_backsolve_kernel<<<1, 1, 0, c->stream>>>(st, L, j);
    if ((rc = ops.update(c->gk_V.p, n, st + L.y(), j, x))) break;
    if (inner && (est_ok || breakdown)) {
      double gj;
      if ((rc = ops.read(st + L.g() + j, &gj, 1))) break;
      status = PRD_OK;
      tr = std::fabs(gj) / beta0 * tr;
      break;
    }
    if (breakdown) {
      if ((rc = op_apply(c, x, w)) || (rc = ops.rsub(b.p, w))) break;
      double rn;
      if ((rc = ops.norm(w, ss, &rn))) break;
      tr = rn / bnorm;
      status = tr < tol ? PRD_OK : PRD_E_BREAKDOWN;
      break;
    }
    tol_in *= 0.5;
  }
  if (!rc && status == PRD_E_NOCONV && !inner) {
    // final true residual
    if (!(rc = op_apply(c, x, w)) && !(rc = ops.rsub(b.p, w))) {
      double rn;
      if (!(rc = ops.norm(w, ss, &rn))) {
        tr = rn / bnorm;
        if (tr < tol) status = PRD_OK;
      }
    }
  }
  if (iters) *iters = it;
  if (true_res) *true_res = tr;
  if (nh_io) *nh_io = nh;
  if (rc) return rc;
  if (status == PRD_E_NOCONV) return fail(c, PRD_E_NOCONV, "GMRES reached max_iter before tol");
  if (status == PRD_E_BREAKDOWN) return fail(c, PRD_E_BREAKDOWN, "GMRES breakdown before tol");
  return PRD_OK;
}

__global__ void d2f_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void f2d_add_kernel(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] += (double)a[i];
}
__global__ void f2d_kernel(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
__global__ void sub_kernel(const double* __restrict__ b, double* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = b[i] - y[i];
}
__global__ void dnorm2_kernel(const double* __restrict__ a, size_t n, double* out) {
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += a[i] * a[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

int apply_operator_acc(Ctx* c, const double* x, double* y, double* ws);
int rhs_acc(Ctx* c, double* b);

static int dnorm(Ctx* c, const double* a, size_t n, double* dsum, double* out) {
  PRD_CUDA_TRY(c, cudaMemsetAsync(dsum, 0, 8, c->stream));
  dnorm2_kernel<<<c->grid_ew(), 256, 0, c->stream>>>(a, n, dsum);
  double h;
  PRD_CUDA_TRY(c, cudaMemcpyAsync(&h, dsum, 8, cudaMemcpyDeviceToHost, c->stream));
  PRD_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *out = std::sqrt(h);
  return PRD_OK;
}

int solve(Ctx* c, double tol, int max_iter, int restart, const void* x0, void* x, int* iters, double* true_res,
          double* hist) {
  const size_t n = nvec(c);
  const size_t vb = n * c->esz;
  int rc;
  if (c->prec == PRD_FP64) {
    DBuf b;
    if ((rc = dalloc(c, b, vb))) return rc;
    if ((rc = rhs(c, b.p))) { dfree(b); return rc; }
    if (x0) PRD_CUDA_TRY(c, cudaMemcpyAsync(x, x0, vb, cudaMemcpyDeviceToDevice, c->stream));
    else PRD_CUDA_TRY(c, cudaMemsetAsync(x, 0, vb, c->stream));
    rc = gmres_core(c, b.p, x, tol, max_iter, restart, iters, true_res, hist, 1.0, nullptr);
    dfree(b);
    return rc;
  }
  // FP32 mode: mixed-precision iterative refinement.  Residuals b - A x are
  // formed with FP64 vectors and FP64 accumulation over the FP32-stored
  // operator (the FP64 residual check); corrections come from FP32 GMRES.
  DBuf b64, x64, r64, ws, d32, r32, dsum;
  auto cleanup = [&]() { dfree(b64); dfree(x64); dfree(r64); dfree(ws); dfree(d32); dfree(r32); dfree(dsum); };
  if ((rc = dalloc(c, b64, n * 8)) || (rc = dalloc(c, x64, n * 8)) || (rc = dalloc(c, r64, n * 8)) ||
      (rc = dalloc(c, ws, 4 * n * 8)) || (rc = dalloc(c, d32, vb)) || (rc = dalloc(c, r32, vb)) ||
      (rc = dalloc(c, dsum, 8))) {
    cleanup();
    return rc;
  }
  const int G = c->grid_ew();
  if ((rc = rhs_acc(c, (double*)b64.p))) { cleanup(); return rc; }
  if (x0) f2d_kernel<<<G, 256, 0, c->stream>>>((const float*)x0, (double*)x64.p, n);
  else PRD_CUDA_TRY(c, cudaMemsetAsync(x64.p, 0, n * 8, c->stream));
  double bn;
  if ((rc = dnorm(c, (const double*)b64.p, n, (double*)dsum.p, &bn))) { cleanup(); return rc; }
  if (!(bn > 0) || !std::isfinite(bn)) { cleanup(); return fail(c, PRD_E_NAN, "right-hand side norm is zero or not finite"); }
  int it_total = 0, nh = 0, status = PRD_E_NOCONV;
  double res = 1.0;
  for (int outer = 0; outer < 12 && it_total < max_iter; ++outer) {
    double rn;
    if (outer == 0 && !x0) {
      // x = 0: the residual is b itself (no FP64 apply)
      PRD_CUDA_TRY(c, cudaMemcpyAsync(r64.p, b64.p, n * 8, cudaMemcpyDeviceToDevice, c->stream));
      rn = bn;
    } else {
      if ((rc = apply_operator_acc(c, (const double*)x64.p, (double*)r64.p, (double*)ws.p))) break;
      sub_kernel<<<G, 256, 0, c->stream>>>((const double*)b64.p, (double*)r64.p, n);
      if ((rc = dnorm(c, (const double*)r64.p, n, (double*)dsum.p, &rn))) break;
    }
    res = rn / bn;
    if (!std::isfinite(res)) { rc = fail(c, PRD_E_NAN, "residual is not finite"); break; }
    if (res < tol) { status = PRD_OK; break; }
    d2f_kernel<<<G, 256, 0, c->stream>>>((const double*)r64.p, (float*)r32.p, n);
    PRD_CUDA_TRY(c, cudaMemsetAsync(d32.p, 0, vb, c->stream));
    const double tin = std::max(0.3 * tol / res, c->refine_floor);
    int its = 0;
    double tr_in = 0;
    const int cap_in = std::min(max_iter - it_total, std::max(2 * restart, 40));
    int rci = gmres_core(c, r32.p, d32.p, tin, cap_in, restart, &its, &tr_in, hist, res, &nh, true);
    it_total += its;
    if (rci && rci != PRD_E_NOCONV) { rc = rci; break; }
    f2d_add_kernel<<<G, 256, 0, c->stream>>>((const float*)d32.p, (double*)x64.p, n);
    PRD_CUDA_TRY(c, cudaPeekAtLastError());
  }
  if (!rc) {
    d2f_kernel<<<G, 256, 0, c->stream>>>((const double*)x64.p, (float*)x, n);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = fail(c, PRD_E_CUDA, cudaGetErrorString(e));
  }
  if (iters) *iters = it_total;
  if (true_res) *true_res = res;
  cleanup();
  if (rc) return rc;
  if (status != PRD_OK) return fail(c, PRD_E_NOCONV, "refined GMRES reached max_iter before tol");
  return PRD_OK;
}

// Adjoint solve A^T lam = g (S13): GMRES in the ctx precision on the FP64
// transposed operator, left-preconditioned with the forward P^-1 (any fixed
// linear map keeps GMRES exact; it only changes the iteration count).
int solve_adjoint(Ctx* c, const void* g, double tol, int max_iter, int restart, void* lam, int* iters,
                  double* true_res, double* hist) {
  PRD_CUDA_TRY(c, cudaMemsetAsync(lam, 0, nvec(c) * c->esz, c->stream));
  c->op_transpose = true;
  const int rc = gmres_core(c, g, lam, tol, max_iter, restart, iters, true_res, hist, 1.0, nullptr);
  c->op_transpose = false;
  return rc;
}

}  // namespace prd
