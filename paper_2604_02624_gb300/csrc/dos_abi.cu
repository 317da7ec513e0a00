// dos_abi.cu - the C ABI of include/dos.h: validation, workspace, launch order.
//
// Launch order of one design step (K layers, all channels, one stream):
//   forward : column pass of gap 0 on the aperture spectrum,
//             K x (row pass [IDFT, crop, checkpoint, Eq. 1 modulation, pad, DFT]
//                  + column pass [DFT, H, IDFT]),
//             output row pass (IDFT of the FOV rows -> o, I = |o|^2)
//   loss    : per-channel statistics, fixed-order total, optional dL/dI
//   backward: seed row pass (2 dL/dI o), K x (adjoint column pass with conj H
//             + adjoint row pass [grad_u, dL/dh partials, conj(t) grad_u]),
//             fixed-order reduction of the partials over channel chunks.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <functional>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/dos.h"
#include "dos_fused.cuh"
#include "dos_gemm.cuh"
#include "dos_internal.h"

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
}  // namespace

namespace dos {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace dos

#define DOS_TIMED(ctx, kind, expr, what)    \
  do {                                      \
    (ctx)->timer.begin((kind), (ctx)->stream); \
    cudaError_t t_ = (expr);                \
    (ctx)->timer.end((ctx)->stream);        \
    DOS_CUDA(t_, what);                     \
  } while (0)

#define DOS_CUDA(expr, what)                                                           \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) return fail(DOS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// CUDA-event timing of each launch, by kernel kind (opt-in).
struct KernelTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Pending { int kind; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  int count[DOS_KERNEL_KINDS] = {0};
  double ms[DOS_KERNEL_KINDS] = {0};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int kind, cudaStream_t s) {
    if (!on) return;
    Pending p{kind, get(), get()};
    cudaEventRecord(p.a, s);
    pending.push_back(p);
  }
  void end(cudaStream_t s) {
    if (!on || pending.empty()) return;
    cudaEventRecord(pending.back().b, s);
  }
  cudaError_t collect() {
    for (const Pending& p : pending) {
      cudaError_t e = cudaEventSynchronize(p.b);
      if (e != cudaSuccess) return e;
      float t = 0.f;
      e = cudaEventElapsedTime(&t, p.a, p.b);
      if (e != cudaSuccess) return e;
      count[p.kind] += 1;
      ms[p.kind] += t;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
    return cudaSuccess;
  }
  void reset() {
    pending.clear();
    for (int k = 0; k < DOS_KERNEL_KINDS; ++k) count[k] = 0, ms[k] = 0;
  }
  void destroy() {
    for (const Pending& p : pending) pool.push_back(p.a), pool.push_back(p.b);
    pending.clear();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

// Multi-pass pass kinds that may run their bulk-prefetching kernels.
constexpr unsigned kBulkCol = 1, kBulkRowFwd = 2, kBulkRowAdj = 4, kBulkAll = 7;

struct dos_ctx {
  KernelTimer timer;
  int n = 0, m = 0, K = 0, nw = 0, nw_total = 0, fov = 0, ap = 0, of = 0, oa = 0, hs = 0;
  int evan = 0, loss = 0, path = DOS_PATH_MULTIPASS;
  int bin = 1;  // detector pixel = bin x bin simulation pixels
  double pitch = 0, n_med = 1, h_base = 0;
  std::vector<double> gaps, lam, nidx, kap;
  std::vector<int> gap_slot;  // gap index -> transfer table slot
  int n_slots = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  const dos::PassOps* ops = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  float2 *S = nullptr, *ckpt = nullptr, *o = nullptr, *Hq = nullptr, *arow = nullptr, *tw = nullptr;
  float2* ckt = nullptr;  // transmission checkpoints of the cluster-resident path
  // create-time input field v1 = P_z0(aperture), [nw][n][n] (Section 2's uniform
  // input field after the first gap; independent of the thickness)
  float2* v1 = nullptr;
  bool ckpt1_is_v1 = false;  // the last multi-pass forward started from v1
  int step_launches = 0;     // kernels in the captured step graph
  dos::ChanConst* chan = nullptr;
  float* partial = nullptr;
  // [K][N][N] thickness of the last forward that saved checkpoints: dos_backward
  // rebuilds t(h) from it, so the caller passes h once per step
  float* h_fwd = nullptr;
  dos::LossStats* stats = nullptr;
  double* d_loss = nullptr;
  double* h_loss = nullptr;  // pinned
  int chunk = 1, n_chunks = 1;
  // multi-pass passes that run their bulk-async prefetching kernels
  // (DOS_PATH_MULTIPASS_BULK: all three; the autotuner may mix them per kind)
  unsigned bulk = 0;

  int* d_err = nullptr;    // set by a kernel whose bounded wait expired
  int* h_err = nullptr;    // pinned copy
  // DOS_INJECT_WAIT_TIMEOUT (tests): the next bulk pass stalls.  1: its copies
  // never arrive, so every block's first wait expires; 2: the copies land, but
  // the odd threads of every block report their first wait as expired; 3 (a
  // column pass): the copies land, but every thread reports its wait for the
  // transfer-table tile of its block's last item as expired
  int inject_stall = 0;
  CUtensorMap tmap_S;        // S as [nw][n][m] 8-byte elements, box {col_group, n, 1}
  CUtensorMap tmap_F;        // the same with box {col_group, fov, 1}: the adjoint's first column pass
  CUtensorMap tmap_H;        // transfer tables as [slots * nw][hs][hs], box {h_box_cols, h_box_rows, 1}
  bool have_tmap = false;     // the bulk column pass runs the plain kernel without them
  int take_stall(unsigned kind) {
    const int v = (bulk & kind) ? inject_stall : 0;
    if (v) inject_stall = 0;
    return v;
  }
  bool have_fwd = false, have_ckpt = false, have_loss = false;
  int launches = 0;
  // cluster-resident path
  std::vector<const dos::FusedOps*> fcands;
  std::vector<int> fcand_clusters;
  const dos::FusedOps* fops = nullptr;
  int n_clusters = 0;
  std::string describe;
  // graph of one design step (dos_step)
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  float* dLdI_step = nullptr;  // [nw][fov][fov] seed buffer of dos_step
  // misaligned layers (Section 3, "vaccination")
  double* d_lam = nullptr;      // wavelengths on the device (kept for the root table)
  float* sq = nullptr;          // signed sqrt(|q|) quadrant table, built on first use
  bool mis_on = false;
  std::vector<float> mis;       // (K+1) x 3 per gap: lateral shift x, y and length change [m]
  long mis_gen = 0;
  dos::Misalign gap_mis(int g) const {
    dos::Misalign m;
    m.sq = mis_on ? sq : nullptr;
    m.df = (float)(1.0 / ((double)this->m * pitch));
    m.ax = mis_on ? mis[3 * g] : 0.f;
    m.ay = mis_on ? mis[3 * g + 1] : 0.f;
    m.dz = mis_on ? mis[3 * g + 2] : 0.f;
    return m;
  }
  // split-BF16 DFT-GEMM path
  dos::GemmPlan gp = {};
  int gchunks = 0;

  template <typename T>
  int alloc(T** p, size_t count, const char* what) {
    void* q = nullptr;
    const size_t b = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, b);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? DOS_ERR_OOM : DOS_ERR_CUDA,
                  std::string("cudaMalloc(") + what + ", " + std::to_string(b) + " bytes): " +
                      cudaGetErrorString(e));
    }
    allocs.push_back(q);
    bytes += b;
    *p = static_cast<T*>(q);
    return DOS_OK;
  }
  void release() {
    cudaStreamSynchronize(stream);
    if (gstream) cudaStreamSynchronize(gstream);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (gstream) cudaStreamDestroy(gstream);
    gexec = nullptr;
    gstream = nullptr;
    ev_in = ev_out = nullptr;
    timer.destroy();
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    if (h_loss) cudaFreeHost(h_loss);
    h_loss = nullptr;
    if (h_err) cudaFreeHost(h_err);
    h_err = nullptr;
  }
  float2* hq_slot(int gap) const { return Hq + (size_t)gap_slot[gap] * nw * hs * hs; }
  dos::PassArgs base() const {
    dos::PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.S = S;
    a.arow = arow;
    a.tw = tw;
    a.chan = chan;
    a.o = o;
    a.n = n;
    a.m = m;
    a.nw = nw;
    a.fov = fov;
    a.of = of;
    a.hs = hs;
    a.chunk = chunk;
    a.n_chunks = n_chunks;
    a.err = d_err;
    a.tmap = have_tmap ? &tmap_S : nullptr;
    a.tmap_rows = n;
    a.hmap = (have_tmap && ops->h_box_cols > 0) ? &tmap_H : nullptr;
    return a;
  }
};

namespace {

bool finite(double x) { return std::isfinite(x); }

int validate(const dos_config* c) {
  if (!c) return fail(DOS_ERR_ARG, "config is NULL");
  if (c->n < 1) return fail(DOS_ERR_ARG, "n must be >= 1");
  if (c->m < c->n) return fail(DOS_ERR_ARG, "m must be >= n");
  if (!dos::pass_ops_for_m(c->m)) {
    int l[32];
    const int k = dos::supported_m_list(l, 32);
    std::string s = "m=" + std::to_string(c->m) + " is not a supported padded size (supported:";
    for (int i = 0; i < k; ++i) s += " " + std::to_string(l[i]);
    return fail(DOS_ERR_ARG, s + ")");
  }
  if (c->n_layers < 1 || c->n_layers > dos::kMaxGaps - 1) return fail(DOS_ERR_ARG, "n_layers must be in [1, 64]");
  if (c->n_lambda < 1 || c->n_lambda > 65535) return fail(DOS_ERR_ARG, "n_lambda must be in [1, 65535]");
  if (c->n_lambda_total != 0 && c->n_lambda_total < c->n_lambda)
    return fail(DOS_ERR_ARG, "n_lambda_total must be 0 or >= n_lambda");
  if (c->fov < 1 || c->fov > c->n || (c->n - c->fov) % 2 != 0)
    return fail(DOS_ERR_ARG, "fov must be in [1, n] with n - fov even");
  const int ap = c->aperture == 0 ? c->fov : c->aperture;
  if (ap < 1 || ap > c->n || (c->n - ap) % 2 != 0)
    return fail(DOS_ERR_ARG, "aperture must be 0 or in [1, n] with n - aperture even");
  if (c->detector_bin < 0 || (c->detector_bin > 1 && c->fov % c->detector_bin != 0))
    return fail(DOS_ERR_ARG, "detector_bin must be 0, 1 or a divisor of fov");
  if (!(c->pitch > 0) || !finite(c->pitch)) return fail(DOS_ERR_ARG, "pitch must be > 0");
  if (!c->gaps || !c->lambda || !c->n_index) return fail(DOS_ERR_ARG, "gaps, lambda and n_index are required");
  for (int i = 0; i <= c->n_layers; ++i)
    if (!(c->gaps[i] >= 0) || !finite(c->gaps[i])) return fail(DOS_ERR_ARG, "gaps must be finite and >= 0");
  for (int w = 0; w < c->n_lambda; ++w) {
    if (!(c->lambda[w] > 0) || !finite(c->lambda[w])) return fail(DOS_ERR_ARG, "lambda must be > 0");
    if (!finite(c->n_index[w])) return fail(DOS_ERR_ARG, "n_index must be finite");
    if (c->kappa && !finite(c->kappa[w])) return fail(DOS_ERR_ARG, "kappa must be finite");
  }
  if (!(c->n_medium > 0) || !finite(c->n_medium)) return fail(DOS_ERR_ARG, "n_medium must be > 0");
  if (!finite(c->h_base)) return fail(DOS_ERR_ARG, "h_base must be finite");
  if (c->evanescent != DOS_EVAN_DECAY && c->evanescent != DOS_EVAN_ZERO)
    return fail(DOS_ERR_ARG, "evanescent must be DOS_EVAN_DECAY or DOS_EVAN_ZERO");
  if (c->loss != DOS_LOSS_MSE && c->loss != DOS_LOSS_MSE_SCALED)
    return fail(DOS_ERR_ARG, "loss must be DOS_LOSS_MSE or DOS_LOSS_MSE_SCALED");
  if (c->path < DOS_PATH_AUTO || c->path > DOS_PATH_DFT_GEMM_X3) return fail(DOS_ERR_ARG, "path must be a DOS_PATH_* value");
  return DOS_OK;
}

int choose_path(dos_ctx* x, int requested);

// Tensor maps of the bulk column pass (elements of 8 bytes: complex64 moved as
// opaque 64-bit words): the row spectra S as [nw][n][m], box {col_group
// columns, n rows, 1 channel} (tmap_S) or {col_group, fov, 1} (tmap_F); the
// transfer tables as [slots * nw][hs][hs] (rows of hs = m/2 + 2 entries, a
// 16-byte multiple), box {h_box_cols, h_box_rows, 1} (tmap_H: whole table rows,
// the quadrant being symmetric), when the column kernel stages an H tile.
// A driver without the entry point leaves the plain column kernel in use.
int make_spectra_map(dos_ctx* x) {
  x->have_tmap = false;
  if (x->n > 256) return DOS_OK;  // one box covers at most 256 rows
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    (void)cudaGetLastError();
    return DOS_OK;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)x->m, (cuuint64_t)x->n, (cuuint64_t)x->nw};
  const cuuint64_t strides[2] = {(cuuint64_t)x->m * 8, (cuuint64_t)x->n * x->m * 8};
  const cuuint32_t estr[3] = {1, 1, 1};
  const int box_rows[2] = {x->n, x->fov};
  CUtensorMap* maps[2] = {&x->tmap_S, &x->tmap_F};
  for (int i = 0; i < 2; ++i) {  // both are encoded, also when fov == n
    const cuuint32_t box[3] = {(cuuint32_t)x->ops->col_group, (cuuint32_t)box_rows[i], 1};
    const CUresult r = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)(
        maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, x->S, dims, strides, box, estr,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(DOS_ERR_CUDA, "cuTensorMapEncodeTiled(row spectra) failed: " + std::to_string((int)r));
  }
  if (x->ops->h_box_cols > 0) {  // the column kernel of this size stages an H tile
    const cuuint64_t hdims[3] = {(cuuint64_t)x->hs, (cuuint64_t)x->hs, (cuuint64_t)x->n_slots * x->nw};
    const cuuint64_t hstrides[2] = {(cuuint64_t)x->hs * 8, (cuuint64_t)x->hs * x->hs * 8};
    const cuuint32_t hbox[3] = {(cuuint32_t)x->ops->h_box_cols, (cuuint32_t)x->ops->h_box_rows, 1};
    const CUresult r = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)(
        &x->tmap_H, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, x->Hq, hdims, hstrides, hbox, estr,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(DOS_ERR_CUDA, "cuTensorMapEncodeTiled(transfer tables) failed: " + std::to_string((int)r));
  }
  x->have_tmap = true;
  return DOS_OK;
}

int build(dos_ctx* x, const dos_config* c) {
  x->n = c->n;
  x->m = c->m;
  x->K = c->n_layers;
  x->nw = c->n_lambda;
  x->nw_total = c->n_lambda_total ? c->n_lambda_total : c->n_lambda;
  x->fov = c->fov;
  x->ap = c->aperture ? c->aperture : c->fov;
  x->of = (c->n - c->fov) / 2;
  x->oa = (c->n - x->ap) / 2;
  // quadrant tables (H depends on fx^2, fy^2): M/2 + 1 frequencies per axis,
  // stored with pitch M/2 + 2 so that a row is a 16-byte multiple (tensor copies)
  x->hs = c->m / 2 + 2;
  x->pitch = c->pitch;
  x->n_med = c->n_medium;
  x->h_base = c->h_base;
  x->evan = c->evanescent;
  x->loss = c->loss;
  x->bin = c->detector_bin > 1 ? c->detector_bin : 1;
  x->path = DOS_PATH_MULTIPASS;
  x->gaps.assign(c->gaps, c->gaps + c->n_layers + 1);
  x->lam.assign(c->lambda, c->lambda + c->n_lambda);
  x->nidx.assign(c->n_index, c->n_index + c->n_lambda);
  x->kap.assign(c->n_lambda, 0.0);
  if (c->kappa) x->kap.assign(c->kappa, c->kappa + c->n_lambda);
  x->ops = dos::pass_ops_for_m(c->m);
  // one transfer table per distinct gap distance
  std::vector<double> slots;
  for (double g : x->gaps) {
    int s = -1;
    for (size_t i = 0; i < slots.size(); ++i)
      if (slots[i] == g) s = (int)i;
    if (s < 0) {
      s = (int)slots.size();
      slots.push_back(g);
    }
    x->gap_slot.push_back(s);
  }
  x->n_slots = (int)slots.size();
  // channel chunks of the adjoint row pass: about 8 blocks per SM in flight
  const int row_blocks = (x->n + x->ops->row_lines - 1) / x->ops->row_lines;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, x->device);
  const int want_chunks = std::max(1, (8 * sms) / std::max(1, row_blocks));
  x->chunk = std::max(1, (x->nw + want_chunks - 1) / want_chunks);
  x->n_chunks = (x->nw + x->chunk - 1) / x->chunk;

  const size_t n2 = (size_t)x->n * x->n;
  // cluster-resident configurations that fit this design
  size_t partial_count = (size_t)x->K * x->n_chunks * n2;
  if (2 * x->n <= x->m) {
    const dos::FusedOps* list[16];
    const int k = dos::fused_ops_for_m(x->m, list, 16);
    for (int i = 0; i < k; ++i) {
      if (list[i]->smem(x->n) > 227 * 1024) continue;
      const int mc = list[i]->max_clusters(x->n);
      if (mc <= 0) continue;
      const int ncl = std::min(mc, x->nw);
      x->fcands.push_back(list[i]);
      x->fcand_clusters.push_back(ncl);
      partial_count = std::max(partial_count, (size_t)ncl * x->K * n2);
    }
  }
  // split-BF16 DFT-GEMM plan (only when requested)
  const bool gemm = c->path == DOS_PATH_DFT_GEMM || c->path == DOS_PATH_DFT_GEMM_X3;
  if (gemm) {
    auto pad = [](int v, int q) { return (v + q - 1) / q * q; };
    x->gp.parts = c->path == DOS_PATH_DFT_GEMM_X3 ? 3 : 2;
    x->gp.n = x->n;
    x->gp.m = x->m;
    x->gp.nwc = std::min(x->nw, 256);
    x->gp.kp1 = pad(2 * x->n, 64);
    x->gp.kp2 = pad(2 * x->m, 64);
    x->gp.rp1 = pad(2 * x->m, 256);
    x->gp.rp2 = pad(2 * x->n, 256);
    x->gchunks = (x->nw + x->gp.nwc - 1) / x->gp.nwc;
    partial_count = std::max(partial_count, (size_t)x->gchunks * x->K * n2);
  }
  int rc;
  if (gemm) {
    dos::GemmPlan& g = x->gp;
    const size_t nwc = (size_t)g.nwc;
    // the data operand holds whole 256-row tiles (the GEMM reads them whole)
    const size_t cm = (nwc * g.m + 255) / 256 * 256, cn = (nwc * g.n + 255) / 256 * 256;
    const size_t xsz = std::max({cm * g.kp1, cm * g.kp2, cn * g.kp1, cn * g.kp2});
    g.F.k = g.G.k = g.X.k = g.Y.k = g.parts;
    for (int q = 0; q < 3; ++q) g.F.p[q] = g.G.p[q] = g.X.p[q] = g.Y.p[q] = nullptr;
    for (int q = 0; q < g.parts; ++q) {
      if ((rc = x->alloc(&g.F.p[q], (size_t)g.rp1 * g.kp1, "DFT matrix"))) return rc;
      if ((rc = x->alloc(&g.G.p[q], (size_t)g.rp2 * g.kp2, "IDFT matrix"))) return rc;
      if ((rc = x->alloc(&g.X.p[q], xsz, "GEMM operand"))) return rc;
      if ((rc = x->alloc(&g.Y.p[q], xsz, "GEMM operand"))) return rc;
    }
    if ((rc = x->alloc(&g.fld, nwc * n2, "GEMM field"))) return rc;
  }
  if ((rc = x->alloc(&x->d_err, 1, "error flag"))) return rc;
  DOS_CUDA(cudaMemsetAsync(x->d_err, 0, sizeof(int), x->stream), "error flag");
  DOS_CUDA(cudaMallocHost(&x->h_err, sizeof(int)), "cudaMallocHost(error flag)");
  *x->h_err = 0;
  if (gemm) {
    x->gp.err = x->d_err;
    DOS_CUDA(dos::launch_build_dft(x->gp, x->stream), "DFT matrices");
  }
  if ((rc = x->alloc(&x->S, (size_t)x->nw * x->n * x->m, "row spectra"))) return rc;
  if ((rc = x->alloc(&x->ckpt, (size_t)x->K * x->nw * n2, "layer checkpoints"))) return rc;
  if (!x->fcands.empty() && (rc = x->alloc(&x->ckt, (size_t)x->K * x->nw * n2, "transmission checkpoints")))
    return rc;
  if ((rc = x->alloc(&x->o, (size_t)x->nw * x->fov * x->fov, "output field"))) return rc;
  if ((rc = x->alloc(&x->Hq, (size_t)x->n_slots * x->nw * x->hs * x->hs, "transfer tables"))) return rc;
  if ((rc = make_spectra_map(x))) return rc;
  if ((rc = x->alloc(&x->arow, (size_t)x->m, "aperture spectrum"))) return rc;
  if ((rc = x->alloc(&x->tw, (size_t)x->ops->Q * dos::twiddle_pitch(x->ops->P), "twiddles"))) return rc;
  if ((rc = x->alloc(&x->chan, (size_t)x->nw, "channel constants"))) return rc;
  if ((rc = x->alloc(&x->partial, partial_count, "gradient partials"))) return rc;
  if ((rc = x->alloc(&x->h_fwd, (size_t)x->K * n2, "saved thickness"))) return rc;
  if ((rc = x->alloc(&x->stats, (size_t)x->nw, "loss statistics"))) return rc;
  if ((rc = x->alloc(&x->d_loss, 1, "loss"))) return rc;
  if ((rc = x->alloc(&x->dLdI_step, (size_t)x->nw * x->fov * x->fov, "step seed"))) return rc;
  DOS_CUDA(cudaMallocHost(&x->h_loss, sizeof(double)), "cudaMallocHost(loss)");

  double *d_lam = nullptr, *d_nidx = nullptr, *d_kap = nullptr;
  if ((rc = x->alloc(&d_lam, (size_t)x->nw, "wavelengths"))) return rc;
  x->d_lam = d_lam;
  if ((rc = x->alloc(&d_nidx, (size_t)x->nw, "indices"))) return rc;
  if ((rc = x->alloc(&d_kap, (size_t)x->nw, "extinction"))) return rc;
  const size_t db = sizeof(double) * x->nw;
  DOS_CUDA(cudaMemcpyAsync(d_lam, x->lam.data(), db, cudaMemcpyHostToDevice, x->stream), "copy lambda");
  DOS_CUDA(cudaMemcpyAsync(d_nidx, x->nidx.data(), db, cudaMemcpyHostToDevice, x->stream), "copy n_index");
  DOS_CUDA(cudaMemcpyAsync(d_kap, x->kap.data(), db, cudaMemcpyHostToDevice, x->stream), "copy kappa");
  DOS_CUDA(dos::launch_chan(x->chan, d_lam, d_nidx, d_kap, x->nw, x->n_med, x->h_base, x->stream),
           "channel constants");
  for (int s = 0; s < x->n_slots; ++s)
    DOS_CUDA(dos::launch_htable(x->Hq + (size_t)s * x->nw * x->hs * x->hs, d_lam, x->nw, slots[s],
                                x->n_med, x->pitch, x->m, x->hs, x->evan, x->stream),
             "transfer tables");
  DOS_CUDA(dos::launch_arow(x->arow, x->m, x->oa, x->ap, x->stream), "aperture spectrum");
  DOS_CUDA(dos::launch_twiddles(x->tw, x->ops->P, x->ops->Q, dos::twiddle_pitch(x->ops->P), x->m, x->stream),
           "twiddles");
  if (!gemm) {
    // v1: the aperture's separable spectrum through gap 0, inverse row DFT, crop
    if ((rc = x->alloc(&x->v1, (size_t)x->nw * n2, "input field"))) return rc;
    dos::PassArgs a = x->base();
    a.Hq = x->hq_slot(0);
    a.out_r0 = 0;
    a.out_r1 = x->n;
    a.fout = x->v1;
    DOS_CUDA(x->ops->col(a, false, true, x->stream), "input field");
    DOS_CUDA(x->ops->row_back(a, x->stream), "input field");
  }
  DOS_CUDA(cudaStreamSynchronize(x->stream), "create");
  if ((rc = choose_path(x, c->path))) return rc;
  DOS_CUDA(cudaStreamSynchronize(x->stream), "create");
  const char* inj = std::getenv("DOS_INJECT_WAIT_TIMEOUT");
  x->inject_stall = (inj && *inj) ? (std::string(inj) == "2"   ? 2
                                     : std::string(inj) == "3" ? 3
                                     : std::string(inj) != "0" ? 1
                                                               : 0)
                                   : 0;
  return DOS_OK;
}

// ------------------------------------------------------------ split-BF16 DFT-GEMM path
// The error flag set by a kernel whose bounded wait expired (tensor-core
// commit or bulk-copy completion), read after the stream has drained.
int flag_after_sync(dos_ctx* c) {
  if (*c->h_err) {
    *c->h_err = 0;
    DOS_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "error flag");
    return fail(DOS_ERR_TIMEOUT, "a bounded wait gave up (mbarrier wait for a tensor-core commit or a bulk copy "
                                 "expired); results of the call are invalid");
  }
  return DOS_OK;
}

int err_check(dos_ctx* c) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DOS_CUDA(cudaStreamIsCapturing(c->stream, &cs), "capture status");
  if (cs != cudaStreamCaptureStatusNone) return DOS_OK;  // checked by the next synchronising call
  DOS_CUDA(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "error flag");
  DOS_CUDA(cudaStreamSynchronize(c->stream), "error flag");
  return flag_after_sync(c);
}

int gemm_check(dos_ctx* c) { return err_check(c); }

int gemm_forward(dos_ctx* c, const float* d_h, float* d_I) {
  dos::GemmPlan& g = c->gp;
  const size_t n2 = (size_t)c->n * c->n, hs2 = (size_t)c->hs * c->hs, f2 = (size_t)c->fov * c->fov;
  c->launches = 0;
  for (int w0 = 0; w0 < c->nw; w0 += g.nwc) {
    const int nc = std::min(g.nwc, c->nw - w0);
    DOS_TIMED(c, DOS_KERNEL_GEMM_FIELD,
              dos::gemm_prep_field(g, nc, nullptr, nullptr, nullptr, nullptr, 2, c->oa, c->ap, c->stream),
              "GEMM aperture field");
    for (int gap = 0; gap <= c->K; ++gap) {
      const bool last = gap == c->K;
      dos::Misalign mg = c->gap_mis(gap);
      if (mg.sq) mg.sq += (size_t)w0 * hs2;
      DOS_TIMED(c, DOS_KERNEL_GEMM_PROPAGATION,
                dos::gemm_propagate(g, nc, c->hq_slot(gap) + (size_t)w0 * hs2, c->hs, false,
                                    last ? c->o + (size_t)w0 * f2 : nullptr,
                                    (last && d_I) ? d_I + (size_t)w0 * f2 : nullptr, c->of, c->fov, mg, &c->launches,
                                    c->stream),
                "GEMM propagation");
      if (!last) {
        DOS_TIMED(c, DOS_KERNEL_GEMM_FIELD,
                  dos::gemm_prep_field(g, nc, g.fld, c->ckpt + ((size_t)gap * c->nw + w0) * n2, d_h + (size_t)gap * n2,
                                       c->chan + w0, 1, 0, 0, c->stream),
                  "GEMM layer modulation");
        ++c->launches;
      }
    }
    c->launches += 1;
  }
  return gemm_check(c);
}

int gemm_backward(dos_ctx* c, const float* d_h, const float* d_dLdI, float* d_dLdh) {
  dos::GemmPlan& g = c->gp;
  const size_t n2 = (size_t)c->n * c->n, hs2 = (size_t)c->hs * c->hs, f2 = (size_t)c->fov * c->fov;
  c->launches = 0;
  int chunk = 0;
  for (int w0 = 0; w0 < c->nw; w0 += g.nwc, ++chunk) {
    const int nc = std::min(g.nwc, c->nw - w0);
    DOS_TIMED(c, DOS_KERNEL_GEMM_FIELD,
              dos::gemm_seed(g, nc, c->o + (size_t)w0 * f2, d_dLdI + (size_t)w0 * f2, c->of, c->fov, c->stream),
              "GEMM adjoint seed");
    DOS_TIMED(c, DOS_KERNEL_GEMM_FIELD,
              dos::gemm_prep_field(g, nc, g.fld, nullptr, nullptr, nullptr, 0, 0, 0, c->stream), "GEMM field");
    c->launches += 2;
    for (int l = c->K; l >= 1; --l) {
      dos::Misalign mg = c->gap_mis(l);
      if (mg.sq) mg.sq += (size_t)w0 * hs2;
      DOS_TIMED(c, DOS_KERNEL_GEMM_PROPAGATION,
                dos::gemm_propagate(g, nc, c->hq_slot(l) + (size_t)w0 * hs2, c->hs, true, nullptr, nullptr, c->of,
                                    c->fov, mg, &c->launches, c->stream),
                "GEMM adjoint propagation");
      DOS_TIMED(c, DOS_KERNEL_GEMM_FIELD,
                dos::gemm_adj_layer(g, nc, c->ckpt + ((size_t)(l - 1) * c->nw + w0) * n2, n2,
                                    d_h + (size_t)(l - 1) * n2, c->chan + w0,
                                    c->partial + ((size_t)chunk * c->K + (l - 1)) * n2, c->stream),
                "GEMM adjoint layer");
      c->launches += 1;
      if (l > 1) {
        DOS_TIMED(c, DOS_KERNEL_GEMM_FIELD,
                  dos::gemm_prep_field(g, nc, g.fld, nullptr, nullptr, nullptr, 0, 0, 0, c->stream), "GEMM field");
        ++c->launches;
      }
    }
  }
  DOS_TIMED(c, DOS_KERNEL_GRAD_REDUCE,
            dos::launch_grad_reduce_flat(c->partial, d_dLdh, c->gchunks, (size_t)c->K * n2, c->stream),
            "gradient reduction");
  ++c->launches;
  return gemm_check(c);
}

// ------------------------------------------------------------ launch sequences
// One kernel launch of a multi-pass sequence: its kind (for the per-kernel
// timer), what it launches on a given stream, and a name for errors.
struct Launch {
  int kind;
  std::function<cudaError_t(cudaStream_t)> go;
  const char* what;
};

// The pass arguments of the channel range [w0, w1): every per-channel array
// starts at channel w0, the tensor-map coordinates are offset by w0.
dos::PassArgs range_args(const dos_ctx* c, int w0, int w1) {
  dos::PassArgs a = c->base();
  a.S = c->S + (size_t)w0 * c->n * c->m;
  a.o = c->o + (size_t)w0 * c->fov * c->fov;
  a.chan = c->chan + w0;
  a.nw = w1 - w0;
  a.n_chunks = (a.nw + c->chunk - 1) / c->chunk;
  a.tmap_w0 = w0;
  return a;
}

// transfer table and displacement table of gap g for the channels from w0
const float2* range_hq(const dos_ctx* c, int g, int w0) { return c->hq_slot(g) + (size_t)w0 * c->hs * c->hs; }
dos::Misalign range_mis(const dos_ctx* c, int g, int w0) {
  dos::Misalign m = c->gap_mis(g);
  if (m.sq) m.sq += (size_t)w0 * c->hs * c->hs;
  return m;
}

// forward: [gap 0 column pass,] K x (row pass + column pass), output row pass
std::vector<Launch> forward_launches(dos_ctx* c, const float* d_h, float* d_I, int save, int w0, int w1) {
  const dos::PassOps* op = c->ops;
  const size_t n2 = (size_t)c->n * c->n;
  std::vector<Launch> L;
  dos::PassArgs a = range_args(c, w0, w1);
  if (!c->ckpt1_is_v1) {
    // the aperture field has the separable spectrum Arow[ky] Arow[kx]
    a.Hq = range_hq(c, 0, w0);
    a.mis = range_mis(c, 0, w0);
    a.out_r0 = 0;
    a.out_r1 = c->n;
    L.push_back({DOS_KERNEL_COLUMN_FORWARD, [op, a](cudaStream_t s) { return op->col(a, false, true, s); },
                 "forward column pass (aperture)"});
  }
  for (int l = 1; l <= c->K; ++l) {
    a.h = d_h + (size_t)(l - 1) * n2;
    a.ckpt = c->ckpt + ((size_t)(l - 1) * c->nw + w0) * n2;
    const bool brow = (c->bulk & kBulkRowFwd) != 0;
    a.stall = c->take_stall(kBulkRowFwd);
    if (l == 1 && c->ckpt1_is_v1) {
      a.fin = c->v1 + (size_t)w0 * n2;
      L.push_back({DOS_KERNEL_ROW_FORWARD,
                   [op, a, brow](cudaStream_t s) { return brow ? op->bulk_row_first(a, s) : op->row_first(a, s); },
                   "first row pass"});
    } else {
      const bool sv = save != 0;
      L.push_back({DOS_KERNEL_ROW_FORWARD,
                   [op, a, brow, sv](cudaStream_t s) { return brow ? op->bulk_row_fwd(a, sv, s) : op->row_fwd(a, sv, s); },
                   "forward row pass"});
    }
    a.Hq = range_hq(c, l, w0);
    a.hmap_z0 = c->gap_slot[l] * c->nw + w0;
    a.mis = range_mis(c, l, w0);
    a.in_r0 = 0;
    a.in_r1 = c->n;
    a.out_r0 = l == c->K ? c->of : 0;
    a.out_r1 = l == c->K ? c->of + c->fov : c->n;
    const bool bcol = (c->bulk & kBulkCol) != 0;
    a.stall = c->take_stall(kBulkCol);
    L.push_back({DOS_KERNEL_COLUMN_FORWARD,
                 [op, a, bcol](cudaStream_t s) { return bcol ? op->bulk_col(a, false, s) : op->col(a, false, false, s); },
                 "forward column pass"});
  }
  a.I = d_I ? d_I + (size_t)w0 * c->fov * c->fov : nullptr;
  L.push_back({DOS_KERNEL_ROW_OUTPUT, [op, a](cudaStream_t s) { return op->row_out(a, s); }, "output row pass"});
  return L;
}

// adjoint: seed row pass, K x (column pass with conj H + row pass); the
// gradient partials of the range's chunks (the caller reduces them)
std::vector<Launch> backward_launches(dos_ctx* c, const float* d_h, const float* d_dLdI, int w0, int w1) {
  const dos::PassOps* op = c->ops;
  const size_t n2 = (size_t)c->n * c->n;
  std::vector<Launch> L;
  dos::PassArgs a = range_args(c, w0, w1);
  a.dLdI = d_dLdI + (size_t)w0 * c->fov * c->fov;
  L.push_back({DOS_KERNEL_ROW_SEED, [op, a](cudaStream_t s) { return op->row_seed(a, s); }, "adjoint seed row pass"});
  for (int l = c->K; l >= 1; --l) {
    a.Hq = range_hq(c, l, w0);
    a.hmap_z0 = c->gap_slot[l] * c->nw + w0;
    a.mis = range_mis(c, l, w0);
    a.in_r0 = l == c->K ? c->of : 0;
    a.in_r1 = l == c->K ? c->of + c->fov : c->n;
    a.tmap = !c->have_tmap ? nullptr : l == c->K ? &c->tmap_F : &c->tmap_S;
    a.tmap_rows = l == c->K ? c->fov : c->n;
    a.out_r0 = 0;
    a.out_r1 = c->n;
    const bool bcol = (c->bulk & kBulkCol) != 0;
    a.stall = c->take_stall(kBulkCol);
    L.push_back({DOS_KERNEL_COLUMN_ADJOINT,
                 [op, a, bcol](cudaStream_t s) { return bcol ? op->bulk_col(a, true, s) : op->col(a, true, false, s); },
                 "adjoint column pass"});
    a.h = d_h + (size_t)(l - 1) * n2;
    a.ckpt = (l == 1 && c->ckpt1_is_v1) ? c->v1 + (size_t)w0 * n2 : c->ckpt + ((size_t)(l - 1) * c->nw + w0) * n2;
    a.partial = c->partial + ((size_t)(l - 1) * c->n_chunks + w0 / c->chunk) * n2;
    const bool brow = (c->bulk & kBulkRowAdj) != 0;
    const bool first = l == 1;
    a.stall = c->take_stall(kBulkRowAdj);
    L.push_back({DOS_KERNEL_ROW_ADJOINT,
                 [op, a, brow, first](cudaStream_t s) { return brow ? op->bulk_row_adj(a, first, s) : op->row_adj(a, first, s); },
                 "adjoint row pass"});
  }
  return L;
}

int enqueue(dos_ctx* c, const Launch& l, cudaStream_t s) {
  c->timer.begin(l.kind, s);
  const cudaError_t e = l.go(s);
  c->timer.end(s);
  DOS_CUDA(e, l.what);
  return DOS_OK;
}

// The launches of one channel range, in order on the context's stream.
int run_launches(dos_ctx* c, const std::vector<Launch>& L) {
  c->launches = (int)L.size();
  for (const Launch& l : L) {
    const int rc = enqueue(c, l, c->stream);
    if (rc) return rc;
  }
  return DOS_OK;
}

int run_forward(dos_ctx* c, const float* d_h, float* d_I, int save) {
  const size_t n2 = (size_t)c->n * c->n;
  c->launches = 0;
  if (save && d_h != c->h_fwd)
    DOS_CUDA(cudaMemcpyAsync(c->h_fwd, d_h, sizeof(float) * c->K * n2, cudaMemcpyDeviceToDevice, c->stream),
             "saved thickness");
  if (c->path == DOS_PATH_DFT_GEMM || c->path == DOS_PATH_DFT_GEMM_X3) return gemm_forward(c, d_h, d_I);
  if (c->path == DOS_PATH_FUSED) {
    dos::FusedArgs f;
    std::memset(&f, 0, sizeof(f));
    f.Hq = c->Hq;
    f.hq_slot_stride = (size_t)c->nw * c->hs * c->hs;
    for (int g = 0; g <= c->K; ++g) f.gap_slot[g] = c->gap_slot[g];
    f.arow = c->arow;
    f.tw = c->tw;
    f.chan = c->chan;
    f.h = d_h;
    f.ckpt = c->ckpt;
    f.ckt = c->ckt;
    c->ckpt1_is_v1 = c->v1 && !c->mis_on;
    f.v1 = c->ckpt1_is_v1 ? c->v1 : nullptr;
    f.o = c->o;
    f.I = d_I;
    f.sq = c->mis_on ? c->sq : nullptr;
    f.df = (float)(1.0 / ((double)c->m * c->pitch));
    for (int g = 0; g <= c->K; ++g) {
      const dos::Misalign mg = c->gap_mis(g);
      f.mis[g][0] = mg.ax;
      f.mis[g][1] = mg.ay;
      f.mis[g][2] = mg.dz;
    }
    f.n = c->n;
    f.nw = c->nw;
    f.K = c->K;
    f.fov = c->fov;
    f.of = c->of;
    f.hs = c->hs;
    f.save = save != 0;
    DOS_TIMED(c, DOS_KERNEL_FUSED_FORWARD, c->fops->launch(f, false, c->n_clusters, c->stream),
              "fused forward sweep");
    c->launches = 1;
    return DOS_OK;
  }
  // gap 0 is the create-time table v1 unless the layers are displaced (then the
  // first gap depends on layer 1's displacement)
  c->ckpt1_is_v1 = c->v1 && !c->mis_on;
  return run_launches(c, forward_launches(c, d_h, d_I, save, 0, c->nw));
}

int run_backward(dos_ctx* c, const float* d_h, const float* d_dLdI, float* d_dLdh) {
  const size_t n2 = (size_t)c->n * c->n;
  c->launches = 0;
  if (c->path == DOS_PATH_DFT_GEMM || c->path == DOS_PATH_DFT_GEMM_X3) return gemm_backward(c, d_h, d_dLdI, d_dLdh);
  if (c->path == DOS_PATH_FUSED) {
    dos::FusedArgs f;
    std::memset(&f, 0, sizeof(f));
    f.Hq = c->Hq;
    f.hq_slot_stride = (size_t)c->nw * c->hs * c->hs;
    for (int g = 0; g <= c->K; ++g) f.gap_slot[g] = c->gap_slot[g];
    f.arow = c->arow;
    f.tw = c->tw;
    f.chan = c->chan;
    f.h = d_h;
    f.ckpt = c->ckpt;
    f.ckt = c->ckt;
    f.v1 = c->ckpt1_is_v1 ? c->v1 : nullptr;
    f.o = c->o;
    f.dLdI = d_dLdI;
    f.sq = c->mis_on ? c->sq : nullptr;
    f.df = (float)(1.0 / ((double)c->m * c->pitch));
    for (int g = 0; g <= c->K; ++g) {
      const dos::Misalign mg = c->gap_mis(g);
      f.mis[g][0] = mg.ax;
      f.mis[g][1] = mg.ay;
      f.mis[g][2] = mg.dz;
    }
    f.partial = c->partial;
    f.n = c->n;
    f.nw = c->nw;
    f.K = c->K;
    f.fov = c->fov;
    f.of = c->of;
    f.hs = c->hs;
    DOS_TIMED(c, DOS_KERNEL_FUSED_ADJOINT, c->fops->launch(f, true, c->n_clusters, c->stream),
              "fused adjoint sweep");
    DOS_TIMED(c, DOS_KERNEL_GRAD_REDUCE,
              dos::launch_grad_reduce_flat(c->partial, d_dLdh, std::min(c->n_clusters, c->nw), (size_t)c->K * n2,
                                           c->stream),
              "gradient reduction");
    c->launches = 2;
    return DOS_OK;
  }
  const int rc = run_launches(c, backward_launches(c, d_h, d_dLdI, 0, c->nw));
  if (rc) return rc;
  DOS_TIMED(c, DOS_KERNEL_GRAD_REDUCE,
            dos::launch_grad_reduce(c->partial, d_dLdh, c->n_chunks, (size_t)c->K * n2, n2, c->stream),
            "gradient reduction");
  ++c->launches;
  return DOS_OK;
}

// ------------------------------------------------------------ autotuner
// Choices of the autotuner: a multi-pass choice -1 - mask, where mask says
// which pass kinds run their bulk-prefetching kernels (kPlain: none, kBulk:
// all), or an index into the cluster-resident candidates.
constexpr int kPlain = -1, kBulk = -1 - (int)kBulkAll;
constexpr int multipass_choice(unsigned mask) { return -1 - (int)mask; }
unsigned choice_mask(int idx) { return (unsigned)(-1 - idx); }

std::string choice_name(const dos_ctx* x, int idx) {
  if (idx < 0) {
    const unsigned b = choice_mask(idx);
    if (b == 0) return "multipass";
    if (b == kBulkAll) return "multipass:bulk";
    std::string s = "multipass:bulk[";
    if (b & kBulkCol) s += "col";
    if (b & kBulkRowFwd) s += std::string(s.back() == '[' ? "" : "+") + "row_fwd";
    if (b & kBulkRowAdj) s += std::string(s.back() == '[' ? "" : "+") + "row_adj";
    return s + "]";
  }
  const dos::FusedOps* f = x->fcands[idx];
  return "fused:C" + std::to_string(f->C) + ":L" + std::to_string(f->lines);
}

std::string tune_key(const dos_ctx* x) {
  cudaDeviceProp p;
  std::string dev = "gpu";
  if (cudaGetDeviceProperties(&p, x->device) == cudaSuccess) dev = std::string(p.name) + "/" + std::to_string(p.multiProcessorCount);
  for (char& ch : dev)
    if (ch == ' ') ch = '_';
  std::ostringstream k;
  k << dev << " n" << x->n << " m" << x->m << " K" << x->K << " w" << x->nw << " f" << x->fov;
  return k.str();
}


void set_choice(dos_ctx* x, int idx) {
  x->bulk = idx < 0 ? choice_mask(idx) : 0;
  if (idx < 0) {
    x->path = x->bulk ? DOS_PATH_MULTIPASS_BULK : DOS_PATH_MULTIPASS;
    x->fops = nullptr;
    x->n_clusters = 0;
  } else {
    x->path = DOS_PATH_FUSED;
    x->fops = x->fcands[idx];
    x->n_clusters = x->fcand_clusters[idx];
  }
}

std::string choice_detail(const dos_ctx* x, int idx) {
  std::ostringstream d;
  d << "path=" << choice_name(x, idx);
  if (idx >= 0)
    d << " threads=" << x->fops->threads << " clusters=" << x->n_clusters << " smem=" << x->fops->smem(x->n);
  return d.str();
}

// time forward(save) + backward of the current choice on zero thickness / zero
// seed; with kind_ms, one more forward + backward with per-launch events gives
// the time of every kernel kind
int time_choice(dos_ctx* x, const float* h0, const float* g0, float* d0, float* ms_out,
                double* kind_ms = nullptr) {
  int rc;
  if ((rc = run_forward(x, h0, nullptr, 1)) || (rc = run_backward(x, h0, g0, d0))) return rc;
  cudaEvent_t a, b;
  DOS_CUDA(cudaEventCreate(&a), "tune event");
  DOS_CUDA(cudaEventCreate(&b), "tune event");
  float best = 1e30f;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(a, x->stream);
    if ((rc = run_forward(x, h0, nullptr, 1)) || (rc = run_backward(x, h0, g0, d0))) break;
    cudaEventRecord(b, x->stream);
    cudaError_t e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e != cudaSuccess) {
      rc = fail(DOS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
      break;
    }
    best = std::min(best, t);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!rc && kind_ms) {
    // the caller's accumulated times survive
    cudaError_t e = x->timer.collect();
    int count0[DOS_KERNEL_KINDS];
    double ms0[DOS_KERNEL_KINDS];
    const bool on0 = x->timer.on;
    for (int k = 0; k < DOS_KERNEL_KINDS; ++k) count0[k] = x->timer.count[k], ms0[k] = x->timer.ms[k];
    x->timer.reset();
    x->timer.on = true;
    if (e == cudaSuccess && !(rc = run_forward(x, h0, nullptr, 1))) rc = run_backward(x, h0, g0, d0);
    if (e == cudaSuccess) e = x->timer.collect();
    if (!rc && e != cudaSuccess) rc = fail(DOS_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
    for (int k = 0; k < DOS_KERNEL_KINDS; ++k) {
      kind_ms[k] = x->timer.ms[k];
      x->timer.count[k] = count0[k];
      x->timer.ms[k] = ms0[k];
    }
    x->timer.on = on0;
  }
  if (!rc) rc = err_check(x);
  *ms_out = best;
  return rc;
}

int choose_path(dos_ctx* x, int requested) {
  if (requested == DOS_PATH_DFT_GEMM || requested == DOS_PATH_DFT_GEMM_X3) {
    x->path = requested;
    x->fops = nullptr;
    x->bulk = 0;
    x->describe = std::string(requested == DOS_PATH_DFT_GEMM_X3 ? "path=dft_gemm_x3" : "path=dft_gemm") +
                  " chunk=" + std::to_string(x->gp.nwc) + " kp=" + std::to_string(x->gp.kp1) + "/" +
                  std::to_string(x->gp.kp2) + " rows=" + std::to_string(x->gp.rp1) + "/" + std::to_string(x->gp.rp2) +
                  (x->gp.parts == 3 ? " (split-BF16, 3 parts, 6 products, tcgen05)" : " (split-BF16, 2 parts, 3 products, tcgen05)");
    return DOS_OK;
  }
  if (requested == DOS_PATH_MULTIPASS) {
    set_choice(x, kPlain);
    x->describe = "path=multipass (requested)";
    return DOS_OK;
  }
  if (requested == DOS_PATH_MULTIPASS_BULK) {
    set_choice(x, kBulk);
    x->describe = "path=multipass:bulk (requested)";
    return DOS_OK;
  }
  if (requested == DOS_PATH_FUSED && x->fcands.empty())
    return fail(DOS_ERR_UNSUPPORTED, "no cluster-resident configuration fits this design (needs n <= m/2 and a "
                                     "compiled configuration for m)");
  // the candidates of the request
  std::vector<int> cands;
  if (requested == DOS_PATH_AUTO) {
    cands.push_back(kPlain);
    cands.push_back(kBulk);
  }
  for (int i = 0; i < (int)x->fcands.size(); ++i) cands.push_back(i);
  if (cands.size() == 1) {
    set_choice(x, cands[0]);
    x->describe = choice_detail(x, cands[0]) + " (only candidate)";
    return DOS_OK;
  }
  // a choice by name: the candidates, and under auto every per-kind mix of
  // plain and bulk-prefetching multi-pass kernels
  auto by_name = [&](const std::string& name, int* out) {
    for (int idx : cands)
      if (choice_name(x, idx) == name) return *out = idx, true;
    if (requested == DOS_PATH_AUTO)
      for (unsigned m = 1; m < kBulkAll; ++m)
        if (choice_name(x, multipass_choice(m)) == name) return *out = multipass_choice(m), true;
    return false;
  };
  // explicit override (profiling, reproducible benchmarks): a name as printed by dos_describe
  const char* force = std::getenv("DOS_FORCE_CONFIG");
  int named = 0;
  if (force && *force && by_name(force, &named)) {
    set_choice(x, named);
    x->describe = choice_detail(x, named) + " (DOS_FORCE_CONFIG)";
    return DOS_OK;
  }
  // cached decision
  const char* cache = std::getenv("DOS_TUNE_CACHE");
  const std::string key = tune_key(x);
  if (cache && *cache) {
    std::ifstream in(cache);
    std::string line;
    while (std::getline(in, line)) {
      if (line.compare(0, key.size() + 1, key + "\t") != 0) continue;
      const std::string v = line.substr(key.size() + 1);
      if (by_name(v, &named)) {
        set_choice(x, named);
        x->describe = choice_detail(x, named) + " (tuning cache)";
        return DOS_OK;
      }
    }
  }
  const size_t n2 = (size_t)x->n * x->n;
  float *h0 = nullptr, *g0 = nullptr, *d0 = nullptr;
  DOS_CUDA(cudaMalloc(&h0, sizeof(float) * x->K * n2), "autotune buffers");
  cudaError_t e = cudaMalloc(&g0, sizeof(float) * (size_t)x->nw * x->fov * x->fov);
  if (e == cudaSuccess) e = cudaMalloc(&d0, sizeof(float) * x->K * n2);
  if (e == cudaSuccess) e = cudaMemsetAsync(h0, 0, sizeof(float) * x->K * n2, x->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g0, 0, sizeof(float) * (size_t)x->nw * x->fov * x->fov, x->stream);
  int rc = DOS_OK;
  if (e != cudaSuccess) rc = fail(DOS_ERR_CUDA, std::string("autotune buffers: ") + cudaGetErrorString(e));
  int best = cands[0];
  float best_ms = 1e30f;
  std::ostringstream d;
  d << "tuned (fwd+bwd ms):";
  // per-kind times of the plain and the bulk-prefetching multi-pass kernels;
  // a mix of the faster of each kind becomes one more candidate
  double kind_plain[DOS_KERNEL_KINDS] = {0}, kind_bulk[DOS_KERNEL_KINDS] = {0};
  for (size_t k = 0; rc == DOS_OK && k < cands.size(); ++k) {
    const int idx = cands[k];
    set_choice(x, idx);
    float ms = 0.f;
    rc = time_choice(x, h0, g0, d0, &ms, idx == kPlain ? kind_plain : idx == kBulk ? kind_bulk : nullptr);
    if (rc) break;
    if (idx == kBulk && requested == DOS_PATH_AUTO) {
      unsigned mix = 0;
      if (kind_bulk[DOS_KERNEL_COLUMN_FORWARD] + kind_bulk[DOS_KERNEL_COLUMN_ADJOINT] <
          kind_plain[DOS_KERNEL_COLUMN_FORWARD] + kind_plain[DOS_KERNEL_COLUMN_ADJOINT])
        mix |= kBulkCol;
      if (kind_bulk[DOS_KERNEL_ROW_FORWARD] < kind_plain[DOS_KERNEL_ROW_FORWARD]) mix |= kBulkRowFwd;
      if (kind_bulk[DOS_KERNEL_ROW_ADJOINT] < kind_plain[DOS_KERNEL_ROW_ADJOINT]) mix |= kBulkRowAdj;
      if (mix != 0 && mix != kBulkAll) cands.insert(cands.begin() + k + 1, multipass_choice(mix));
    }
    d << " " << choice_name(x, idx);
    if (idx >= 0) d << "x" << x->fcand_clusters[idx];
    d << "=" << ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = idx;
    }
  }
  cudaFree(h0);
  cudaFree(g0);
  cudaFree(d0);
  if (rc) return rc;
  set_choice(x, best);
  x->describe = choice_detail(x, best) + " | " + d.str();
  if (cache && *cache) {
    std::ofstream out(cache, std::ios::app);
    out << key << "\t" << choice_name(x, best) << "\n";
  }
  return DOS_OK;
}

int check_ctx(dos_ctx* c) {
  if (!c) return fail(DOS_ERR_ARG, "context is NULL");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return fail(DOS_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  return DOS_OK;
}

}  // namespace

extern "C" {

DOS_API int dos_supported_m(int* out, int cap) {
  int tmp[64];
  const int k = dos::supported_m_list(tmp, 64);
  for (int i = 0; out && i < k && i < cap; ++i) out[i] = tmp[i];
  return k;
}

DOS_API int dos_create(dos_ctx** out, const dos_config* cfg, void* cuda_stream) {
  if (!out) return fail(DOS_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate(cfg);
  if (rc) return rc;
  dos_ctx* x = new (std::nothrow) dos_ctx();
  if (!x) return fail(DOS_ERR_OOM, "host allocation of the context failed");
  x->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&x->device);
  if (e != cudaSuccess) {
    delete x;
    return fail(DOS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  rc = build(x, cfg);
  if (rc) {
    const std::string keep = g_err;
    x->release();
    delete x;
    g_err = keep;
    return rc;
  }
  *out = x;
  return DOS_OK;
}

DOS_API int dos_set_stream(dos_ctx* c, void* cuda_stream) {
  int rc = check_ctx(c);
  if (rc) return rc;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return DOS_OK;
}

DOS_API int dos_forward(dos_ctx* c, const float* d_h, float* d_I, int save_for_backward) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!d_h) return fail(DOS_ERR_ARG, "d_h is NULL");
  c->have_fwd = c->have_ckpt = c->have_loss = false;
  if ((rc = run_forward(c, d_h, d_I, save_for_backward))) return rc;
  c->have_fwd = true;
  c->have_ckpt = save_for_backward != 0;
  return DOS_OK;
}

DOS_API int dos_loss(dos_ctx* c, const float* d_T, double* h_loss, float* d_psnr, float* d_dLdI) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_fwd) return fail(DOS_ERR_STATE, "dos_loss needs a dos_forward first");
  if (!d_T) return fail(DOS_ERR_ARG, "d_T is NULL");
  const int det2 = (c->fov / c->bin) * (c->fov / c->bin);
  const double norm = (double)c->nw_total * det2;
  c->launches = 0;
  DOS_TIMED(c, DOS_KERNEL_LOSS,
            dos::launch_loss_stats(c->o, d_T, c->stats, c->nw, c->fov, c->bin, d_dLdI, norm, c->loss, c->stream),
            "loss statistics and dL/dI");
  DOS_TIMED(c, DOS_KERNEL_LOSS, dos::launch_loss_final(c->stats, c->nw, det2, norm, c->loss, c->d_loss, d_psnr, c->stream),
            "loss total");
  c->launches += 2;
  c->have_loss = true;
  if (h_loss) return dos_read_loss(c, h_loss);
  return DOS_OK;
}

DOS_API int dos_set_misalignment(dos_ctx* c, const double* disp) {
  int rc = check_ctx(c);
  if (rc) return rc;
  ++c->mis_gen;
  if (!disp) {
    c->mis_on = false;
    return DOS_OK;
  }
  for (int i = 0; i < 3 * c->K; ++i)
    if (!std::isfinite(disp[i])) return fail(DOS_ERR_ARG, "displacements must be finite");
  if (!c->sq) {
    if ((rc = c->alloc(&c->sq, (size_t)c->nw * c->hs * c->hs, "root table"))) return rc;
    DOS_CUDA(dos::launch_sqtable(c->sq, c->d_lam, c->nw, c->n_med, c->pitch, c->m, c->hs, c->stream), "root table");
  }
  // layer l (1..K) displaced by D_l; planes 0 (aperture) and K+1 (detector) fixed:
  // gap g carries the lateral shift D_g - D_{g+1} and the length change dz_{g+1} - dz_g
  c->mis.assign(3 * (c->K + 1), 0.f);
  auto D = [&](int l, int k) { return (l >= 1 && l <= c->K) ? disp[3 * (l - 1) + k] : 0.0; };
  for (int g = 0; g <= c->K; ++g) {
    c->mis[3 * g] = (float)(D(g, 0) - D(g + 1, 0));
    c->mis[3 * g + 1] = (float)(D(g, 1) - D(g + 1, 1));
    c->mis[3 * g + 2] = (float)(D(g + 1, 2) - D(g, 2));
  }
  c->mis_on = true;
  return DOS_OK;
}

DOS_API int dos_efficiency(dos_ctx* c, float* d_eta) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_fwd) return fail(DOS_ERR_STATE, "dos_efficiency needs a dos_forward first");
  if (!d_eta) return fail(DOS_ERR_ARG, "d_eta is NULL");
  DOS_CUDA(dos::launch_efficiency(c->o, d_eta, c->nw, c->fov * c->fov, c->ap, c->stream), "efficiency");
  c->launches = 1;
  return DOS_OK;
}

DOS_API int dos_quantize_thickness(const float* d_h, float* d_hq, size_t count, double h_max, int bits,
                                   void* cuda_stream) {
  if (!d_h || !d_hq) return fail(DOS_ERR_ARG, "d_h and d_hq are required");
  if (!(h_max > 0) || !std::isfinite(h_max)) return fail(DOS_ERR_ARG, "h_max must be > 0");
  if (bits < 1 || bits > 24) return fail(DOS_ERR_ARG, "bits must be in [1, 24]");
  if (count == 0) return DOS_OK;
  DOS_CUDA(dos::launch_quantize(d_h, d_hq, count, h_max, bits, static_cast<cudaStream_t>(cuda_stream)), "quantize");
  return DOS_OK;
}

DOS_API int dos_read_loss(dos_ctx* c, double* h_loss) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_loss) return fail(DOS_ERR_STATE, "no loss computed yet");
  if (!h_loss) return fail(DOS_ERR_ARG, "h_loss is NULL");
  DOS_CUDA(cudaMemcpyAsync(c->h_loss, c->d_loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
           "read loss");
  DOS_CUDA(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "error flag");
  DOS_CUDA(cudaStreamSynchronize(c->stream), "read loss");
  *h_loss = *c->h_loss;
  return flag_after_sync(c);
}

DOS_API int dos_backward(dos_ctx* c, const float* d_dLdI, float* d_dLdh) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_ckpt) return fail(DOS_ERR_STATE, "dos_backward needs dos_forward(save_for_backward=1) first");
  if (!d_dLdI || !d_dLdh) return fail(DOS_ERR_ARG, "d_dLdI and d_dLdh are required");
  return run_backward(c, c->h_fwd, d_dLdI, d_dLdh);
}

DOS_API int dos_step(dos_ctx* c, const float* d_h, const float* d_T, float* d_dLdh, float* d_I, float* d_psnr,
                     double* h_loss) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!d_h || !d_T || !d_dLdh) return fail(DOS_ERR_ARG, "d_h, d_T and d_dLdh are required");
  if (!c->gstream) {
    DOS_CUDA(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking), "step stream");
    DOS_CUDA(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming), "step event");
    DOS_CUDA(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming), "step event");
  }
  const void* key[6] = {d_h, d_T, d_dLdh, d_I, d_psnr, reinterpret_cast<const void*>(c->mis_gen)};
  bool same = c->gexec != nullptr;
  for (int i = 0; i < 6; ++i) same = same && key[i] == c->gkey[i];
  DOS_CUDA(cudaEventRecord(c->ev_in, c->stream), "step order");
  DOS_CUDA(cudaStreamWaitEvent(c->gstream, c->ev_in, 0), "step order");
  if (!same) {
    const bool timing = c->timer.on;
    const int inject = c->inject_stall;  // an injected stall never enters the graph
    c->timer.on = false;
    c->inject_stall = 0;
    cudaStream_t user = c->stream;
    c->stream = c->gstream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      const int det2 = (c->fov / c->bin) * (c->fov / c->bin);
      const double norm = (double)c->nw_total * det2;
      rc = run_forward(c, d_h, d_I, 1);
      const int fwd_launches = c->launches;
      if (!rc)
        e = dos::launch_loss_stats(c->o, d_T, c->stats, c->nw, c->fov, c->bin, c->dLdI_step, norm, c->loss,
                                   c->gstream);
      if (!rc && e == cudaSuccess)
        e = dos::launch_loss_final(c->stats, c->nw, det2, norm, c->loss, c->d_loss, d_psnr, c->gstream);
      if (!rc && e == cudaSuccess) rc = run_backward(c, d_h, c->dLdI_step, d_dLdh);
      if (!rc) c->step_launches = fwd_launches + 2 + c->launches;
      cudaError_t e2 = cudaStreamEndCapture(c->gstream, &g);
      if (e == cudaSuccess) e = e2;
    }
    c->stream = user;
    c->timer.on = timing;
    c->inject_stall = inject;
    if (rc || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (rc) return rc;
      return fail(DOS_ERR_CUDA, std::string("step capture: ") + cudaGetErrorString(e));
    }
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(DOS_ERR_CUDA, std::string("step instantiate: ") + cudaGetErrorString(e));
    for (int i = 0; i < 6; ++i) c->gkey[i] = key[i];
  }
  DOS_CUDA(cudaGraphLaunch(c->gexec, c->gstream), "step graph launch");
  DOS_CUDA(cudaEventRecord(c->ev_out, c->gstream), "step order");
  DOS_CUDA(cudaStreamWaitEvent(c->stream, c->ev_out, 0), "step order");
  c->launches = c->step_launches;
  c->have_fwd = c->have_ckpt = c->have_loss = true;
  if (h_loss) return dos_read_loss(c, h_loss);
  return DOS_OK;
}

DOS_API int dos_output_field(dos_ctx* c, float* d_o) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_fwd) return fail(DOS_ERR_STATE, "no forward yet");
  if (!d_o) return fail(DOS_ERR_ARG, "d_o is NULL");
  DOS_CUDA(cudaMemcpyAsync(d_o, c->o, sizeof(float2) * c->nw * c->fov * c->fov, cudaMemcpyDeviceToDevice,
                           c->stream),
           "copy output field");
  return DOS_OK;
}

DOS_API int dos_layer_field(dos_ctx* c, int layer, float* d_v) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (!c->have_ckpt) return fail(DOS_ERR_STATE, "no forward with save_for_backward yet");
  if (layer < 1 || layer > c->K) return fail(DOS_ERR_ARG, "layer must be in [1, n_layers]");
  if (!d_v) return fail(DOS_ERR_ARG, "d_v is NULL");
  const size_t n2 = (size_t)c->n * c->n;
  const bool table = layer == 1 && c->ckpt1_is_v1 &&
                     (c->path == DOS_PATH_MULTIPASS || c->path == DOS_PATH_MULTIPASS_BULK || c->path == DOS_PATH_FUSED);
  DOS_CUDA(cudaMemcpyAsync(d_v, table ? c->v1 : c->ckpt + (size_t)(layer - 1) * c->nw * n2,
                           sizeof(float2) * c->nw * n2, cudaMemcpyDeviceToDevice, c->stream),
           "copy layer field");
  return DOS_OK;
}

DOS_API int dos_propagate(dos_ctx* c, int gap, const float* d_in, float* d_out, int adjoint) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (gap < 0 || gap > c->K) return fail(DOS_ERR_ARG, "gap must be in [0, n_layers]");
  if (!d_in || !d_out || d_in == d_out) return fail(DOS_ERR_ARG, "d_in and d_out must be distinct non-NULL");
  const dos::PassOps* op = c->ops;
  c->launches = 0;
  c->have_fwd = c->have_ckpt = c->have_loss = false;  // the spectra buffer is reused
  dos::PassArgs a = c->base();
  a.fin = reinterpret_cast<const float2*>(d_in);
  a.fout = reinterpret_cast<float2*>(d_out);
  a.Hq = c->hq_slot(gap);
  a.mis = c->gap_mis(gap);
  a.in_r0 = 0;
  a.in_r1 = c->n;
  a.out_r0 = 0;
  a.out_r1 = c->n;
  DOS_CUDA(op->row_in(a, c->stream), "propagate row pass");
  DOS_CUDA(op->col(a, adjoint != 0, false, c->stream), "propagate column pass");
  DOS_CUDA(op->row_back(a, c->stream), "propagate back row pass");
  c->launches = 3;
  return DOS_OK;
}

DOS_API int dos_set_timing(dos_ctx* c, int enable) {
  int rc = check_ctx(c);
  if (rc) return rc;
  c->timer.reset();
  c->timer.on = enable != 0;
  return DOS_OK;
}

DOS_API int dos_kernel_time(dos_ctx* c, int kind, int* launches, double* ms) {
  int rc = check_ctx(c);
  if (rc) return rc;
  if (kind < 0 || kind >= DOS_KERNEL_KINDS) return fail(DOS_ERR_ARG, "unknown kernel kind");
  DOS_CUDA(c->timer.collect(), "kernel timing");
  if (launches) *launches = c->timer.count[kind];
  if (ms) *ms = c->timer.ms[kind];
  return DOS_OK;
}

DOS_API size_t dos_workspace_bytes(const dos_ctx* c) { return c ? c->bytes : 0; }

DOS_API int dos_last_launch_count(const dos_ctx* c) { return c ? c->launches : 0; }

DOS_API int dos_path(const dos_ctx* c) { return c ? c->path : 0; }

DOS_API int dos_describe(const dos_ctx* c, char* buf, int cap) {
  const std::string d = c ? c->describe : std::string();
  if (buf && cap > 0) {
    const size_t k = std::min((size_t)cap - 1, d.size());
    std::memcpy(buf, d.data(), k);
    buf[k] = 0;
  }
  return (int)d.size();
}

DOS_API void dos_destroy(dos_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  c->release();
  delete c;
}

DOS_API const char* dos_last_error(const dos_ctx* c) {
  (void)c;  // the message is the calling thread's: a failed dos_create has no context to hold it
  return g_err.c_str();
}

}  // extern "C"
