// C ABI of libkmv: argument checks, work-item tables, workspace and dispatch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "kmv_internal.cuh"
#include "kmv_tc.cuh"

using namespace kmv;

namespace kmv {
const char* points_error(const kmv_points* pts, int32_t chains) {
  if (!pts) return "points is NULL";
  if (pts->n_inst < 1) return "n_inst must be >= 1";
  if (!pts->offsets) return "offsets is NULL";
  if (pts->d < 1 || pts->d > kMaxD) return "d must be in [1, 64]";
  if (pts->ard != 0 && pts->ard != 1) return "ard must be 0 or 1";
  if (chains < 1 || chains > 65535) return "chains must be in [1, 65535]";
  if (pts->offsets[0] != 0) return "offsets[0] must be 0";
  for (int b = 0; b < pts->n_inst; ++b)
    if (pts->offsets[b + 1] < pts->offsets[b]) return "offsets must be non-decreasing";
  const int64_t n = pts->offsets[pts->n_inst];
  if (n > (int64_t(1) << 40)) return "too many rows";
  if (n > 0 && !pts->x) return "x is NULL";
  if ((int64_t)pts->n_inst * chains > (int64_t(1) << 30)) return "too many systems";
  if (pts->cheb < 0 || pts->cheb > kMaxChebOrder) return "cheb must be in [0, 32]";
  if (pts->cheb > 1 && pts->d > kMaxChebDims) return "cheb >= 2 needs d <= 8";
  if (pts->cheb > 0 && cheb_n_coef(pts->cheb, pts->d) < 0) return "cheb^d must be <= 1024";
  return nullptr;
}
}  // namespace kmv

namespace {

kmv_status fail(kmv_handle h, kmv_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  return s;
}

#define KMV_CUDA(h, expr)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(h, KMV_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)

#define KMV_TRY(expr)                 \
  do {                                \
    kmv_status s_ = (expr);           \
    if (s_ != KMV_OK) return s_;      \
  } while (0)

// Bump allocator over the handle workspace; 256-byte aligned regions.
constexpr int kMaxPoles = 32;

struct Arena {
  size_t used = 0;
  size_t take(size_t bytes) {
    const size_t off = used;
    used += (bytes + 255) & ~size_t(255);
    return off;
  }
};

kmv_status reserve(kmv_handle h, size_t bytes) {
  if (bytes <= h->ws_bytes) return KMV_OK;
  if (h->capturing)
    return fail(h, KMV_EINVAL,
                "workspace would grow during stream capture: make the same call once before capturing");
  if (h->ws) {
    KMV_CUDA(h, cudaDeviceSynchronize());
    KMV_CUDA(h, cudaFree(h->ws));
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  const size_t want = bytes + bytes / 4 + (1 << 20);
  if (cudaMalloc(&h->ws, want) != cudaSuccess) {
    cudaGetLastError();
    h->ws = nullptr;
    return fail(h, KMV_ENOMEM, "workspace allocation of " + std::to_string(want) + " bytes failed");
  }
  h->ws_bytes = want;
  return KMV_OK;
}

template <class T>
T* at(kmv_handle h, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(h->ws) + off);
}

kmv_status check_points(kmv_handle h, const kmv_points* pts, int32_t chains) {
  if (!h) return KMV_EINVAL;
  const char* e = points_error(pts, chains);
  return e ? fail(h, KMV_EINVAL, e) : KMV_OK;
}

// Builds (or reuses) the row-tile work items of this point set on the device.
kmv_status prepare_layout(kmv_handle h, const kmv_points* pts, int32_t chains, cudaStream_t st) {
  KMV_CUDA(h, cudaSetDevice(h->device));
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  KMV_CUDA(h, cudaStreamIsCapturing(st, &cs));
  h->capturing = cs != cudaStreamCaptureStatusNone;
  Layout& L = h->layout;
  const int n_inst = pts->n_inst;
  const bool same = h->cached_d == pts->d && (int)h->cached_offsets.size() == n_inst + 1 &&
                    std::equal(h->cached_offsets.begin(), h->cached_offsets.end(), pts->offsets);
  L.chains = chains;
  L.d = pts->d;
  L.ard = pts->ard;
  L.cheb = pts->cheb;
  L.n_coef = pts->cheb > 0 ? cheb_n_coef(pts->cheb, pts->d) : 0;
  L.n_theta_int = 2 + (pts->ard ? pts->d : 1);
  L.n_theta = L.cheb ? L.n_coef + L.n_theta_int - 1 : L.n_theta_int;
  if (same) return KMV_OK;
  if (h->capturing)
    return fail(h, KMV_EINVAL, "new point layout during stream capture: make the same call once before capturing");

  L.n_inst = n_inst;
  L.offsets.assign(pts->offsets, pts->offsets + n_inst + 1);
  L.n_total = L.offsets[n_inst];
  L.item_inst.clear();
  L.item_row0.clear();
  L.inst_item0.assign(n_inst + 1, 0);
  L.max_items_per_inst = 0;
  for (int b = 0; b < n_inst; ++b) {
    L.inst_item0[b] = (int32_t)L.item_inst.size();
    const int64_t nb = L.offsets[b + 1] - L.offsets[b];
    const int64_t tiles = (nb + kTile - 1) / kTile;
    for (int64_t t = 0; t < tiles; ++t) {
      L.item_inst.push_back(b);
      L.item_row0.push_back(L.offsets[b] + t * kTile);
    }
    L.max_items_per_inst = std::max<int>(L.max_items_per_inst, (int)tiles);
  }
  L.inst_item0[n_inst] = (int32_t)L.item_inst.size();
  L.n_items = (int)L.item_inst.size();
  if ((int64_t)L.item_inst.size() > (int64_t(1) << 30)) return fail(h, KMV_EINVAL, "too many tiles");

  const size_t b_off = sizeof(int64_t) * (n_inst + 1);
  const size_t b_inst = sizeof(int32_t) * std::max(1, L.n_items);
  const size_t b_row0 = sizeof(int64_t) * std::max(1, L.n_items);
  const size_t b_ii = sizeof(int32_t) * (n_inst + 1);
  const size_t o_off = 0, o_row0 = (b_off + 255) & ~size_t(255);
  const size_t o_inst = o_row0 + ((b_row0 + 255) & ~size_t(255));
  const size_t o_ii = o_inst + ((b_inst + 255) & ~size_t(255));
  const size_t total = o_ii + b_ii;
  if (total > h->tables_bytes) {
    if (h->tables) {
      KMV_CUDA(h, cudaDeviceSynchronize());
      KMV_CUDA(h, cudaFree(h->tables));
      h->tables = nullptr;
      h->tables_bytes = 0;
    }
    if (cudaMalloc(&h->tables, total) != cudaSuccess) {
      cudaGetLastError();
      h->tables = nullptr;
      return fail(h, KMV_ENOMEM, "table allocation failed");
    }
    h->tables_bytes = total;
  }
  // The tables are staged through host memory that outlives the copy: wait for it.
  char* base = static_cast<char*>(h->tables);
  KMV_CUDA(h, cudaMemcpyAsync(base + o_off, L.offsets.data(), b_off, cudaMemcpyHostToDevice, st));
  if (L.n_items) {
    KMV_CUDA(h, cudaMemcpyAsync(base + o_row0, L.item_row0.data(), sizeof(int64_t) * L.n_items,
                                cudaMemcpyHostToDevice, st));
    KMV_CUDA(h, cudaMemcpyAsync(base + o_inst, L.item_inst.data(), sizeof(int32_t) * L.n_items,
                                cudaMemcpyHostToDevice, st));
  }
  KMV_CUDA(h, cudaMemcpyAsync(base + o_ii, L.inst_item0.data(), b_ii, cudaMemcpyHostToDevice, st));
  KMV_CUDA(h, cudaStreamSynchronize(st));
  h->dev.offsets = reinterpret_cast<const int64_t*>(base + o_off);
  h->dev.item_row0 = reinterpret_cast<const int64_t*>(base + o_row0);
  h->dev.item_inst = reinterpret_cast<const int32_t*>(base + o_inst);
  h->dev.inst_item0 = reinterpret_cast<const int32_t*>(base + o_ii);
  h->cached_offsets = L.offsets;
  h->cached_d = pts->d;
  return KMV_OK;
}

KmvArgs base_args(kmv_handle h, const kmv_points* pts, const double* theta) {
  KmvArgs a{};
  a.L = h->dev;
  a.chains = h->layout.chains;
  a.d = pts->d;
  a.ard = pts->ard;
  a.n_theta = h->layout.n_theta;
  a.n_total = h->layout.n_total;
  a.x = pts->x;
  a.theta = theta;
  a.n_z = 1;
  if (h->layout.cheb) {
    // the Chebyshev family runs as the stationary kernel between amplitudes,
    // prepared from this theta by cheb_prepare
    a.theta = h->cheb_theta;
    a.n_theta = h->layout.n_theta_int;
    a.amp = h->cheb_amp;
  }
  return a;
}

// For the Chebyshev family: the internal stationary parameters and the per-point
// amplitudes exp(C_theta(x)) of theta (user layout), plus the backward's scratch
// for up to m_bwd columns.  A no-op for the SE kernel.
kmv_status cheb_prepare(kmv_handle h, const kmv_points* pts, const double* theta, int m_bwd, cudaStream_t st) {
  const Layout& L = h->layout;
  if (!L.cheb) return KMV_OK;
  const size_t n_sys = (size_t)L.n_inst * L.chains;
  const size_t vec = (size_t)L.chains * std::max<int64_t>(1, L.n_total);
  const size_t items = (size_t)std::max(1, L.n_items) * L.chains;
  Arena ar;
  const size_t o_th = ar.take(sizeof(double) * n_sys * L.n_theta_int);
  const size_t o_amp = ar.take(sizeof(float) * vec);
  const size_t o_gi = ar.take(sizeof(double) * n_sys * L.n_theta_int);
  const size_t o_pt = ar.take(sizeof(double) * items * L.n_coef);
  const size_t o_kv = ar.take(sizeof(float) * vec * std::max(1, m_bwd));
  const size_t o_kg = ar.take(sizeof(float) * vec * std::max(1, m_bwd));
  if (ar.used > h->cheb_bytes) {
    if (h->capturing)
      return fail(h, KMV_EINVAL, "workspace would grow during stream capture: make the same call once before capturing");
    if (h->cheb_buf) {
      KMV_CUDA(h, cudaDeviceSynchronize());
      KMV_CUDA(h, cudaFree(h->cheb_buf));
      h->cheb_buf = nullptr;
      h->cheb_bytes = 0;
    }
    if (cudaMalloc(&h->cheb_buf, ar.used) != cudaSuccess) {
      cudaGetLastError();
      h->cheb_buf = nullptr;
      return fail(h, KMV_ENOMEM, "amplitude buffer allocation failed");
    }
    h->cheb_bytes = ar.used;
  }
  char* base = static_cast<char*>(h->cheb_buf);
  h->cheb_theta = reinterpret_cast<double*>(base + o_th);
  h->cheb_amp = reinterpret_cast<float*>(base + o_amp);
  h->cheb_gint = reinterpret_cast<double*>(base + o_gi);
  h->cheb_part = reinterpret_cast<double*>(base + o_pt);
  h->cheb_kv = reinterpret_cast<float*>(base + o_kv);
  h->cheb_kg = reinterpret_cast<float*>(base + o_kg);
  h->cheb_mcap = std::max(1, m_bwd);
  KMV_CUDA(h, launch_cheb_prepare(h->dev, L.n_items, (int)n_sys, L.chains, L.n_total, L.d, L.cheb, L.n_coef,
                                  L.n_theta, L.n_theta_int, pts->x, theta, h->cheb_theta, h->cheb_amp, st));
  return KMV_OK;
}

// --- building blocks used by several entry points -------------------------------------

// The FP32 forward, with its J range split over more CTAs when one CTA per
// (item, chain, column chunk) would leave most SMs idle (forward_jsplit).
kmv_status simt_forward(kmv_handle h, const KmvArgs& a, cudaStream_t st) {
  const Layout& L = h->layout;
  if (L.n_items == 0) return KMV_OK;
  if ((a.cg_sys || a.ms_sys) && !(a.m == 1 && a.dot_partial))
    return fail(h, KMV_EINVAL, "internal: fused CG step needs the one-column product");
  const int js = forward_jsplit(L.n_items, L.chains, a.m, (int64_t)L.max_items_per_inst * kTile, h->num_sms);
  if (js > 1) {
    const size_t need = sizeof(double) * (size_t)js * L.chains * (size_t)L.n_total * a.m;
    if (need > h->simt_part_bytes) {
      if (h->capturing)
        return fail(h, KMV_EINVAL, "FP32 forward scratch not prepared: make the same call once before capturing");
      if (h->simt_part) cudaFree(h->simt_part);
      h->simt_part = nullptr;
      h->simt_part_bytes = 0;
      if (cudaMalloc(&h->simt_part, need) != cudaSuccess) {
        cudaGetLastError();
        h->simt_part = nullptr;
        return fail(h, KMV_ENOMEM, "FP32 forward scratch allocation failed");
      }
      h->simt_part_bytes = need;
    }
  }
  KMV_CUDA(h, launch_forward_simt(a, L.n_items, js, h->simt_part, st));
  return KMV_OK;
}

kmv_status run_forward(kmv_handle h, const KmvArgs& a, kmv_precision prec, cudaStream_t st) {
  if (h->layout.n_items == 0) return KMV_OK;
  if (prec == KMV_BF16_HILO) {
    kmv_status s = tc_forward(h, a, st);
    return s;
  }
  {
    ProfScope prof(h, KMV_KERNEL_FORWARD, st);
    KMV_TRY(simt_forward(h, a, st));
  }
  return KMV_OK;
}

size_t backward_ws_bytes(const Layout& L, int m) {
  const int mp = backward_mp(m);
  const int nz = (m + mp - 1) / mp;
  return sizeof(double) * (size_t)std::max(1, L.n_items) * L.chains * nz * L.n_theta;
}

kmv_status run_backward_stationary(kmv_handle h, KmvArgs a, double* grad, double* partial,
                                   kmv_precision prec, cudaStream_t st) {
  const Layout& L = h->layout;
  if (prec == KMV_BF16_HILO) {
    // shapes outside the tensor-core adjoint's range (d > 32, or operand
    // tiles that do not fit in tensor or shared memory) use the FP32 adjoint
    const kmv_status s = tc_backward(h, a, grad, st);
    if (s != KMV_EUNSUPPORTED) return s;
  }
  const int mp = backward_mp(a.m);
  a.n_z = (a.m + mp - 1) / mp;
  a.grad_partial = partial;
  if (L.n_items > 0) {
    ProfScope prof(h, KMV_KERNEL_ADJOINT, st);
    KMV_CUDA(h, launch_backward_simt(a, L.n_items, st));
  }
  KMV_CUDA(h, launch_grad_finalize(h->dev, L.n_inst, L.chains, a.n_theta, L.ard, L.d, a.n_z,
                                   a.theta, partial, grad, st));
  return KMV_OK;
}

// Adjoint of sum G o (A V) with args from base_args; grad in the caller's theta layout.
// For the Chebyshev family the stationary adjoint (with amplitudes) gives the
// lengthscale and noise entries, and the Theta entries are sum_i T_t(x_i) h_i with
// h = G o (K V) + V o (K G) summed over columns (K without the noise term).
kmv_status run_backward(kmv_handle h, KmvArgs a, double* grad, double* partial,
                        kmv_precision prec, cudaStream_t st) {
  const Layout& L = h->layout;
  if (!L.cheb) return run_backward_stationary(h, a, grad, partial, prec, st);
  if (a.m > h->cheb_mcap) return fail(h, KMV_EINVAL, "internal: amplitude scratch prepared for fewer columns");
  KMV_TRY(run_backward_stationary(h, a, h->cheb_gint, partial, prec, st));
  KmvArgs f = a;
  f.G = nullptr;
  f.col_shift = nullptr;
  f.Y64 = nullptr;
  f.dot_partial = nullptr;
  f.grad_partial = nullptr;
  f.no_diag = 1;
  f.V = a.V;
  f.Y = h->cheb_kv;
  KMV_TRY(run_forward(h, f, prec, st));
  f.V = a.G;
  f.Y = h->cheb_kg;
  KMV_TRY(run_forward(h, f, prec, st));
  KMV_CUDA(h, launch_cheb_grad(h->dev, L.n_items, L.n_inst, L.chains, L.n_total, L.d, L.cheb, L.n_coef, L.n_theta,
                               L.n_theta_int, a.m, a.x, a.V, a.G, h->cheb_kv, h->cheb_kg, a.sys_active,
                               h->cheb_part, h->cheb_gint, grad, st));
  return KMV_OK;
}

// While `st` is being captured: records the loop `while (*n_active > 0)
// body(stream)` as a conditional WHILE node, so that a replayed solve stops
// when its systems have converged, as the eager loop does.  The first test
// is a kernel captured before the node; the body ends with the next test.
// The body is captured on the handle's side stream into the node's graph.
template <class Body>
kmv_status capture_while(kmv_handle h, cudaStream_t st, const int32_t* n_active, Body&& body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  KMV_CUDA(h, cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) return fail(h, KMV_EINVAL, "internal: capture_while outside a capture");
  cudaGraphConditionalHandle cond;
  KMV_CUDA(h, cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
  KMV_CUDA(h, launch_loop_cond(cond, n_active, st));
  const cudaGraphNode_t* deps = nullptr;
  size_t n_deps = 0;
  KMV_CUDA(h, cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &n_deps));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  KMV_CUDA(h, cudaGraphAddNode(&node, g, deps, nullptr, n_deps, &np));
  cudaGraph_t body_graph = np.conditional.phGraph_out[0];
  KMV_CUDA(h, cudaStreamBeginCaptureToGraph(h->side, body_graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  kmv_status s = body(h->side);
  if (s == KMV_OK && launch_loop_cond(cond, n_active, h->side) != cudaSuccess) s = KMV_ECUDA;
  cudaGraph_t captured = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->side, &captured);
  if (s != KMV_OK) return s;
  KMV_CUDA(h, e);
  KMV_CUDA(h, cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return KMV_OK;
}

struct CgBufs {
  float *r, *p, *q;
  double *partial, *partial2;
  CgSys* sys;
  int32_t *active, *n_active;
  uint32_t* count;   // 2 n_sys counters of the fused iteration (p.q step, r.r step)
};

size_t cg_layout(const Layout& L, Arena& ar, size_t off[8]) {
  const size_t vec = sizeof(float) * (size_t)L.chains * std::max<int64_t>(1, L.n_total);
  const size_t items = (size_t)std::max(1, L.n_items) * L.chains;
  const size_t n_sys = (size_t)L.n_inst * L.chains;
  off[0] = ar.take(vec);
  off[1] = ar.take(vec);
  off[2] = ar.take(vec);
  off[3] = ar.take(sizeof(double) * items);
  off[4] = ar.take(sizeof(double) * items * 2);
  off[5] = ar.take(sizeof(CgSys) * n_sys);
  off[6] = ar.take(sizeof(int32_t) * n_sys);
  off[7] = ar.take(sizeof(int32_t) * 4 + sizeof(uint32_t) * 2 * n_sys);
  return ar.used;
}

CgBufs cg_bufs(kmv_handle h, const size_t off[8]) {
  CgBufs b;
  b.r = at<float>(h, off[0]);
  b.p = at<float>(h, off[1]);
  b.q = at<float>(h, off[2]);
  b.partial = at<double>(h, off[3]);
  b.partial2 = at<double>(h, off[4]);
  b.sys = at<CgSys>(h, off[5]);
  b.active = at<int32_t>(h, off[6]);
  b.n_active = at<int32_t>(h, off[7]);
  b.count = reinterpret_cast<uint32_t*>(b.n_active + 4);
  return b;
}

// Batched CG on A(theta_s) x = rhs (Sec. 3.2.1 primitive (1)); see kmv_cg_solve.
kmv_status run_cg(kmv_handle h, const kmv_points* pts, const double* theta, const float* rhs,
                  int64_t rhs_stride, float* x, double tol, int maxiter, int warm,
                  int32_t* status, int32_t* iters, const CgBufs& B, kmv_precision prec,
                  cudaStream_t st) {
  const Layout& L = h->layout;
  const int n_sys = L.n_inst * L.chains;
  KmvArgs a = base_args(h, pts, theta);
  a.m = 1;
  if (warm) {
    a.V = x;
    a.Y = B.q;
    KMV_TRY(run_forward(h, a, prec, st));
  }
  if (L.n_items > 0)
    KMV_CUDA(h, launch_cg_init(h->dev, L.n_items, L.chains, L.n_total, rhs, rhs_stride, B.q, x, B.r,
                               B.p, warm, B.partial2, st));
  KMV_CUDA(h, launch_cg_reduce_init(h->dev, L.n_inst, L.chains, B.partial2, tol, B.sys, B.active,
                                    B.n_active, st));
  const int check_every = 4;
  a.V = B.p;
  a.Y = B.q;
  a.sys_active = B.active;
  a.dot_partial = B.partial;
  // An iteration needs no separate reduction launches: the product's epilogue
  // takes each system's p.q step in the CTA that finishes the system last, and
  // the x, r update takes the r.r step likewise, with the same per-system
  // arithmetic in the same order as the separate kernels.  With the
  // tensor-core one-column product (KMV_BF16_HILO where it takes the FMA-pipe
  // form) the product also forms p = r + beta p before its tiles; the FP32
  // product reads p from every CTA, so there the direction update stays a
  // kernel at the end of the iteration.
  const bool tc_fma = prec == KMV_BF16_HILO && x_width_fma_ok(pts->d);
  const bool fused = L.n_items > 0 && (tc_fma || prec == KMV_FP32);
  if (fused) {
    KMV_CUDA(h, cudaMemsetAsync(B.count, 0, sizeof(uint32_t) * 2 * n_sys, st));
    a.cg_sys = B.sys;
    a.cg_active = B.active;
    a.cg_n_active = B.n_active;
    a.cg_count = B.count;
    a.cg_r = B.r;
  }
  // one CG iteration on every active system; theta is fixed within the solve,
  // so the products after the first reuse its operand tiles
  auto iteration = [&](cudaStream_t s, int reuse) -> kmv_status {
    a.reuse_prep = reuse;
    KMV_TRY(run_forward(h, a, prec, s));
    if (fused) {
      KMV_CUDA(h, launch_cg_update_xr_rr(h->dev, L.n_items, L.chains, L.n_total, B.sys, B.active, x, B.r, B.p,
                                         B.q, B.partial, B.count + n_sys, tol, maxiter, B.n_active, s));
      if (!tc_fma)
        KMV_CUDA(h, launch_cg_update_p(h->dev, L.n_items, L.chains, L.n_total, B.sys, B.active, B.r, B.p, s));
      return KMV_OK;
    }
    KMV_CUDA(h, launch_cg_reduce_pq(h->dev, L.n_inst, L.chains, B.partial, B.sys, B.active, s));
    KMV_CUDA(h, launch_cg_update_xr(h->dev, L.n_items, L.chains, L.n_total, B.sys, B.active, x, B.r,
                                    B.p, B.q, B.partial, s));
    KMV_CUDA(h, launch_cg_reduce_rr(h->dev, L.n_inst, L.chains, B.partial, tol, maxiter, B.sys,
                                    B.active, B.n_active, s));
    KMV_CUDA(h, launch_cg_update_p(h->dev, L.n_items, L.chains, L.n_total, B.sys, B.active, B.r,
                                   B.p, s));
    return KMV_OK;
  };
  if (h->capturing) {
    // Under stream capture: the first iteration (which prepares the operand
    // tiles; on systems already converged it changes nothing), then a WHILE
    // node repeating iterations while any system is active, so a replay stops
    // at convergence (or at maxiter, which deactivates a system) like the eager loop.
    if (maxiter > 0) {
      KMV_TRY(iteration(st, warm ? 1 : 0));
      KMV_TRY(capture_while(h, st, B.n_active, [&](cudaStream_t s2) { return iteration(s2, 1); }));
    }
  } else {
    for (int it = 0; it < maxiter; ++it) {
      if (it % check_every == 0) {
        KMV_CUDA(h, cudaMemcpyAsync(h->host_flag, B.n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        KMV_CUDA(h, cudaStreamSynchronize(st));
        if (*h->host_flag == 0) break;
      }
      KMV_TRY(iteration(st, (it > 0 || warm) ? 1 : 0));
    }
  }
  KMV_CUDA(h, launch_cg_finish(n_sys, B.sys, status, iters, st));
  return KMV_OK;
}

// --- preconditioned CG (randomized Nystrom, set by kmv_set_preconditioner) -----------

struct PcgBufs {
  float *r, *p, *q, *z;
  double *partial, *partial2, *prz, *proj, *coef;
  PcgSys* sys;
  int32_t *active, *n_active;
};

void pcg_layout(const Layout& L, int rank, Arena& ar, size_t off[12]) {
  const size_t vec = sizeof(float) * (size_t)L.chains * std::max<int64_t>(1, L.n_total);
  const size_t items = (size_t)std::max(1, L.n_items) * L.chains;
  const size_t n_sys = (size_t)L.n_inst * L.chains;
  for (int k = 0; k < 4; ++k) off[k] = ar.take(vec);
  off[4] = ar.take(sizeof(double) * items);
  off[5] = ar.take(sizeof(double) * items * 2);
  off[6] = ar.take(sizeof(double) * items);
  off[7] = ar.take(sizeof(double) * items * rank);
  off[8] = ar.take(sizeof(double) * n_sys * rank);
  off[9] = ar.take(sizeof(PcgSys) * n_sys);
  off[10] = ar.take(sizeof(int32_t) * n_sys);
  off[11] = ar.take(sizeof(int32_t) * 4);
}

PcgBufs pcg_bufs(kmv_handle h, const size_t off[12]) {
  PcgBufs b;
  b.r = at<float>(h, off[0]);
  b.p = at<float>(h, off[1]);
  b.q = at<float>(h, off[2]);
  b.z = at<float>(h, off[3]);
  b.partial = at<double>(h, off[4]);
  b.partial2 = at<double>(h, off[5]);
  b.prz = at<double>(h, off[6]);
  b.proj = at<double>(h, off[7]);
  b.coef = at<double>(h, off[8]);
  b.sys = at<PcgSys>(h, off[9]);
  b.active = at<int32_t>(h, off[10]);
  b.n_active = at<int32_t>(h, off[11]);
  return b;
}

// Batched preconditioned CG on A(theta_s) x = rhs with the handle's preconditioner;
// arguments and stopping rule as run_cg (under capture: exactly maxiter masked iterations).
kmv_status run_pcg(kmv_handle h, const kmv_points* pts, const double* theta, const float* rhs, int64_t rhs_stride,
                   float* x, double tol, int maxiter, int warm, int32_t* status, int32_t* iters, const PcgBufs& B,
                   kmv_precision prec, cudaStream_t st) {
  const Layout& L = h->layout;
  const int n_sys = L.n_inst * L.chains;
  const PcgPrecond P{h->pc.rank, h->pc.U, h->pc.lam};
  KmvArgs a = base_args(h, pts, theta);
  a.m = 1;
  if (warm) {
    a.V = x;
    a.Y = B.q;
    KMV_TRY(run_forward(h, a, prec, st));
  }
  KMV_CUDA(h, launch_pcg_init(h->dev, L.n_items, L.chains, L.n_total, rhs, rhs_stride, B.q, x, B.r, warm,
                              B.partial2, st));
  KMV_CUDA(h, launch_pcg_precond(h->dev, L.n_items, L.n_inst, L.chains, L.n_total, P, a.theta, a.n_theta, B.r, B.z,
                                 nullptr, B.proj, B.coef, B.prz, st));
  KMV_CUDA(h, cudaMemsetAsync(B.n_active, 0, sizeof(int32_t), st));
  KMV_CUDA(h, launch_pcg_setup(h->dev, L.n_inst, L.chains, B.partial2, B.prz, tol, B.sys, B.active, B.n_active, st));
  const size_t vbytes = sizeof(float) * (size_t)L.chains * L.n_total;
  if (vbytes) KMV_CUDA(h, cudaMemcpyAsync(B.p, B.z, vbytes, cudaMemcpyDeviceToDevice, st));
  a.V = B.p;
  a.Y = B.q;
  a.sys_active = B.active;
  a.dot_partial = B.partial;
  const int check_every = 4;
  auto iteration = [&](cudaStream_t s, int reuse) -> kmv_status {
    a.reuse_prep = reuse;
    KMV_TRY(run_forward(h, a, prec, s));
    KMV_CUDA(h, launch_pcg_alpha(h->dev, L.n_inst, L.chains, B.partial, B.sys, B.active, s));
    KMV_CUDA(h, launch_pcg_update_xr(h->dev, L.n_items, L.chains, L.n_total, B.sys, B.active, x, B.r, B.p, B.q,
                                     B.partial, s));
    KMV_CUDA(h, launch_pcg_precond(h->dev, L.n_items, L.n_inst, L.chains, L.n_total, P, a.theta, a.n_theta, B.r,
                                   B.z, B.active, B.proj, B.coef, B.prz, s));
    KMV_CUDA(h, cudaMemsetAsync(B.n_active, 0, sizeof(int32_t), s));
    KMV_CUDA(h, launch_pcg_beta(h->dev, L.n_inst, L.chains, B.partial, B.prz, tol, maxiter, B.sys, B.active,
                                B.n_active, s));
    KMV_CUDA(h, launch_pcg_update_p(h->dev, L.n_items, L.chains, L.n_total, B.sys, B.active, B.z, B.p, s));
    return KMV_OK;
  };
  if (h->capturing) {
    // as in run_cg: one iteration, then a WHILE node until no system is active
    if (maxiter > 0) {
      KMV_TRY(iteration(st, warm ? 1 : 0));
      KMV_TRY(capture_while(h, st, B.n_active, [&](cudaStream_t s2) { return iteration(s2, 1); }));
    }
  } else {
    for (int it = 0; it < maxiter; ++it) {
      if (it % check_every == 0) {
        KMV_CUDA(h, cudaMemcpyAsync(h->host_flag, B.n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        KMV_CUDA(h, cudaStreamSynchronize(st));
        if (*h->host_flag == 0) break;
      }
      KMV_TRY(iteration(st, (it > 0 || warm) ? 1 : 0));
    }
  }
  KMV_CUDA(h, launch_pcg_finish(n_sys, B.sys, B.active, status, iters, st));
  return KMV_OK;
}

// Extra buffers of the refined (KMV_BF16_HILO) solve.
struct RefineBufs {
  float *q32, *r, *dx, *pdummy;
  double *partial2, *prev_rr;
  CgSys* sys;
  int32_t *active, *n_active, *in_status, *in_iters;
};

void refine_layout(const Layout& L, Arena& ar, size_t off[11]) {
  const size_t vec = sizeof(float) * (size_t)L.chains * std::max<int64_t>(1, L.n_total);
  const size_t items = (size_t)std::max(1, L.n_items) * L.chains;
  const size_t n_sys = (size_t)L.n_inst * L.chains;
  off[0] = ar.take(vec);
  off[1] = ar.take(vec);
  off[2] = ar.take(vec);
  off[3] = ar.take(vec);
  off[4] = ar.take(sizeof(double) * items * 2);
  off[5] = ar.take(sizeof(CgSys) * n_sys);
  off[6] = ar.take(sizeof(int32_t) * n_sys);
  off[7] = ar.take(sizeof(double) * 2);   // n_active (int32) + worst rr/bb (double at +8)
  off[8] = ar.take(sizeof(int32_t) * n_sys);
  off[9] = ar.take(sizeof(int32_t) * n_sys);
  off[10] = ar.take(sizeof(double) * n_sys);
}

RefineBufs refine_bufs(kmv_handle h, const size_t off[11]) {
  RefineBufs b;
  b.q32 = at<float>(h, off[0]);
  b.r = at<float>(h, off[1]);
  b.dx = at<float>(h, off[2]);
  b.pdummy = at<float>(h, off[3]);
  b.partial2 = at<double>(h, off[4]);
  b.sys = at<CgSys>(h, off[5]);
  b.active = at<int32_t>(h, off[6]);
  b.n_active = at<int32_t>(h, off[7]);
  b.in_status = at<int32_t>(h, off[8]);
  b.in_iters = at<int32_t>(h, off[9]);
  b.prev_rr = at<double>(h, off[10]);
  return b;
}

// Solve with the KMV_BF16_HILO operator to FP32 accuracy by iterative
// refinement (Carson & Higham's mixed-precision scheme): the true residual
// r = rhs - A x is formed with the FP32 operator, the correction A dx = r is
// solved by CG with the tensor-core operator, and x += dx, until
// ||r|| <= tol ||rhs|| or the residual stops falling (the FP32 floor).  The
// inner tolerance is 1e-5 when the product takes the FMA-pipe path with the
// three-way exponent split (relative operator error ~1e-6), else 1e-3.
// Returns the summed inner iterations.
kmv_status run_cg_refined(kmv_handle h, const kmv_points* pts, const double* theta, const float* rhs,
                          int64_t rhs_stride, float* x, double tol, int maxiter, int warm, int32_t* status,
                          int32_t* iters, const CgBufs& B, const RefineBufs& R, const PcgBufs* PB,
                          cudaStream_t st) {
  const Layout& L = h->layout;
  const int n_sys = L.n_inst * L.chains;
  const int64_t nvec = (int64_t)L.chains * L.n_total;
  // the tensor-core operator's relative accuracy bounds how far a correction is worth solving
  const double floor_tol = x_width_fma_ok(pts->d) ? 1e-5 : 1e-3;
  double* worst = reinterpret_cast<double*>(reinterpret_cast<char*>(R.n_active) + 8);
  const int max_outer = 12;
  const int kCaptureOuter = 3;
  if (!warm && nvec > 0) KMV_CUDA(h, cudaMemsetAsync(x, 0, sizeof(float) * nvec, st));
  KMV_CUDA(h, cudaMemsetAsync(status, 0, sizeof(int32_t) * n_sys, st));
  if (iters) KMV_CUDA(h, cudaMemsetAsync(iters, 0, sizeof(int32_t) * n_sys, st));
  KmvArgs a = base_args(h, pts, theta);
  a.m = 1;
  for (int outer = 0; outer <= max_outer; ++outer) {
    // r = rhs - A x with the FP32 operator; active = ||r|| > tol ||rhs||
    a.V = x;
    a.Y = R.q32;
    KMV_TRY(simt_forward(h, a, st));
    if (L.n_items > 0)
      KMV_CUDA(h, launch_cg_init(h->dev, L.n_items, L.chains, L.n_total, rhs, rhs_stride, R.q32, x, R.r,
                                 R.pdummy, 1, R.partial2, st));
    KMV_CUDA(h, launch_cg_reduce_init(h->dev, L.n_inst, L.chains, R.partial2, tol, R.sys, R.active, R.n_active,
                                      st));
    KMV_CUDA(h, launch_refine_stagnation(n_sys, outer, R.sys, R.prev_rr, R.active, R.n_active, worst, st));
    double inner_tol = floor_tol;
    if (h->capturing) {
      // no host check under capture: a fixed number of refinement steps
      if (outer == kCaptureOuter) break;
    } else {
      KMV_CUDA(h, cudaMemcpyAsync(h->host_flag, R.n_active, 16, cudaMemcpyDeviceToHost, st));
      KMV_CUDA(h, cudaStreamSynchronize(st));
      if (*h->host_flag == 0 || outer == max_outer) break;
      // solve the correction only as far as the target needs: ||r|| must fall to tol ||rhs||
      double wr;
      std::memcpy(&wr, reinterpret_cast<const char*>(h->host_flag) + 8, sizeof(double));
      const double ratio = wr > 0.0 ? std::sqrt(wr) : 1.0;
      inner_tol = std::min(0.5, std::max(floor_tol, 0.5 * tol / ratio));
    }
    // correction from the tensor-core operator, on the systems still active
    if (L.n_items > 0) KMV_CUDA(h, launch_mask_rows(h->dev, L.n_items, L.chains, L.n_total, R.active, R.r, st));
    if (PB)
      KMV_TRY(run_pcg(h, pts, theta, R.r, L.n_total, R.dx, inner_tol, maxiter, 0, R.in_status, R.in_iters, *PB,
                      KMV_BF16_HILO, st));
    else
      KMV_TRY(run_cg(h, pts, theta, R.r, L.n_total, R.dx, inner_tol, maxiter, 0, R.in_status, R.in_iters, B,
                     KMV_BF16_HILO, st));
    KMV_CUDA(h, launch_axpy(nvec, R.dx, x, st));
    KMV_CUDA(h, launch_refine_merge(n_sys, R.in_status, R.in_iters, status, iters, st));
  }
  KMV_CUDA(h, launch_refine_finish(n_sys, R.active, R.sys, tol, status, st));
  return KMV_OK;
}

// Buffers of a solve in either precision, with or without the preconditioner.
struct SolveLayout {
  size_t cg[8];
  size_t rf[11];
  size_t pcg[12];
  bool refined, pc;
};

void solve_layout(kmv_handle h, Arena& ar, kmv_precision prec, SolveLayout& S) {
  const Layout& L = h->layout;
  cg_layout(L, ar, S.cg);
  // The single-column tensor-core product (three-way split exponent, FP32 P.v)
  // is as accurate as the FP32 form, so the BF16 form solves with it directly;
  // only shapes without that product (d > 17) solve by refinement.
  S.refined = prec == KMV_BF16_HILO && !x_width_fma_ok(L.d);
  if (S.refined) refine_layout(L, ar, S.rf);
  S.pc = h->pc_on;
  if (S.pc) pcg_layout(L, h->pc.rank, ar, S.pcg);
}

kmv_status run_solve(kmv_handle h, const kmv_points* pts, const double* theta, const float* rhs, int64_t rhs_stride,
                     float* x, double tol, int maxiter, int warm, int32_t* status, int32_t* iters,
                     const SolveLayout& S, kmv_precision prec, cudaStream_t st) {
  const Layout& L = h->layout;
  if (S.pc && (h->pc.n_inst != L.n_inst || h->pc.chains != L.chains || h->pc.n_total != L.n_total))
    return fail(h, KMV_EINVAL, "the preconditioner was built for another layout (n_inst, chains, N_total)");
  PcgBufs pb;
  if (S.pc) pb = pcg_bufs(h, S.pcg);
  if (S.refined)
    return run_cg_refined(h, pts, theta, rhs, rhs_stride, x, tol, maxiter, warm, status, iters, cg_bufs(h, S.cg),
                          refine_bufs(h, S.rf), S.pc ? &pb : nullptr, st);
  if (S.pc) return run_pcg(h, pts, theta, rhs, rhs_stride, x, tol, maxiter, warm, status, iters, pb, prec, st);
  return run_cg(h, pts, theta, rhs, rhs_stride, x, tol, maxiter, warm, status, iters, cg_bufs(h, S.cg), prec, st);
}

// --- multi-column CG: the shifted systems of the pole expansion ---------------------

struct McgBufs {
  float *r, *p, *q;
  double *partial, *partial2;
  McgCol* cols;
  int32_t *sys_any, *n_active;
};

void mcg_layout(const Layout& L, int m, Arena& ar, size_t off[8]) {
  const size_t vec = sizeof(float) * (size_t)L.chains * std::max<int64_t>(1, L.n_total) * m;
  const size_t items = (size_t)std::max(1, L.n_items) * L.chains * m;
  const size_t n_sys = (size_t)L.n_inst * L.chains;
  off[0] = ar.take(vec);
  off[1] = ar.take(vec);
  off[2] = ar.take(vec);
  off[3] = ar.take(sizeof(double) * items);
  off[4] = ar.take(sizeof(double) * items * 2);
  off[5] = ar.take(sizeof(McgCol) * n_sys * m);
  off[6] = ar.take(sizeof(int32_t) * n_sys);
  off[7] = ar.take(sizeof(double) * 2);   // n_active (int32) + worst rr/bb (double at +8)
}

McgBufs mcg_bufs(kmv_handle h, const size_t off[8]) {
  McgBufs b;
  b.r = at<float>(h, off[0]);
  b.p = at<float>(h, off[1]);
  b.q = at<float>(h, off[2]);
  b.partial = at<double>(h, off[3]);
  b.partial2 = at<double>(h, off[4]);
  b.cols = at<McgCol>(h, off[5]);
  b.sys_any = at<int32_t>(h, off[6]);
  b.n_active = at<int32_t>(h, off[7]);
  return b;
}

// Preconditioner of the multi-column CG: the handle's Nystrom factors, applied per
// column with mu_q = sigma^2 + shift_q (the Woodbury form for each shifted system).
struct McgPre {
  PcgPrecond P;
  float* z;
  double *proj, *coef, *prz;
};

void mcg_pre_layout(const Layout& L, int m, int rank, Arena& ar, size_t off[4]) {
  const size_t vec = sizeof(float) * (size_t)L.chains * std::max<int64_t>(1, L.n_total) * m;
  const size_t items = (size_t)std::max(1, L.n_items) * L.chains * m;
  off[0] = ar.take(vec);
  off[1] = ar.take(sizeof(double) * items * rank);
  off[2] = ar.take(sizeof(double) * (size_t)L.n_inst * L.chains * m * rank);
  off[3] = ar.take(sizeof(double) * items);
}

McgPre mcg_pre(kmv_handle h, const size_t off[4]) {
  McgPre p;
  p.P = PcgPrecond{h->pc.rank, h->pc.U, h->pc.lam};
  p.z = at<float>(h, off[0]);
  p.proj = at<double>(h, off[1]);
  p.coef = at<double>(h, off[2]);
  p.prz = at<double>(h, off[3]);
  return p;
}

// CG on (A(theta_s) + shift[s m + q] I) x_q = b_q for the m columns q of every
// system s, one m-column product per iteration; the column results stay in B.cols.
// b is (chains, N) shared by the columns (b_cols == 0) or (chains, N, m).  With
// pre, each column runs preconditioned CG.
kmv_status run_mcg(kmv_handle h, const kmv_points* pts, const double* theta, const float* shifts, int m,
                   const float* b, int b_cols, float* x, double tol, int maxiter, int warm, const McgBufs& B,
                   kmv_precision prec, cudaStream_t st, const McgPre* pre = nullptr) {
  const Layout& L = h->layout;
  KmvArgs a = base_args(h, pts, theta);
  a.m = m;
  a.col_shift = shifts;
  a.col_shift_stride = m;
  if (warm) {
    a.V = x;
    a.Y = B.q;
    KMV_TRY(run_forward(h, a, prec, st));
  }
  KMV_CUDA(h, launch_mcg_init(h->dev, L.n_items, L.chains, L.n_total, m, b, b_cols, B.q, warm, x, B.r, B.p,
                              B.partial2, st));
  KMV_CUDA(h, cudaMemsetAsync(B.n_active, 0, sizeof(int32_t), st));
  KMV_CUDA(h, launch_mcg_reduce_init(h->dev, L.n_inst, L.chains, m, B.partial2, tol, B.cols, B.sys_any,
                                     B.n_active, st));
  const size_t vbytes = sizeof(float) * (size_t)L.chains * L.n_total * m;
  if (pre) {
    KMV_CUDA(h, launch_mcg_precond(h->dev, L.n_items, L.n_inst, L.chains, L.n_total, m, pre->P, a.theta, a.n_theta,
                                   shifts, B.r, pre->z, B.sys_any, pre->proj, pre->coef, pre->prz, st));
    KMV_CUDA(h, launch_mcg_set_rz(h->dev, L.n_inst, L.chains, m, pre->prz, B.cols, st));
    if (vbytes) KMV_CUDA(h, cudaMemcpyAsync(B.p, pre->z, vbytes, cudaMemcpyDeviceToDevice, st));
  }
  a.V = B.p;
  a.Y = B.q;
  a.sys_active = B.sys_any;
  const int check_every = 4;
  for (int it = 0; it < maxiter; ++it) {
    if (it % check_every == 0) {
      KMV_CUDA(h, cudaMemcpyAsync(h->host_flag, B.n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      KMV_CUDA(h, cudaStreamSynchronize(st));
      if (*h->host_flag == 0) break;
    }
    KMV_TRY(run_forward(h, a, prec, st));
    KMV_CUDA(h, launch_mcg_dot(h->dev, L.n_items, L.chains, L.n_total, m, B.p, B.q, B.sys_any, B.partial, st));
    KMV_CUDA(h, launch_mcg_alpha(h->dev, L.n_inst, L.chains, m, B.partial, B.cols, B.sys_any, pre ? 1 : 0, st));
    KMV_CUDA(h, launch_mcg_update_xr(h->dev, L.n_items, L.chains, L.n_total, m, B.cols, B.sys_any, x, B.r, B.p,
                                     B.q, B.partial, st));
    if (pre)
      KMV_CUDA(h, launch_mcg_precond(h->dev, L.n_items, L.n_inst, L.chains, L.n_total, m, pre->P, a.theta,
                                     a.n_theta, shifts, B.r, pre->z, B.sys_any, pre->proj, pre->coef, pre->prz, st));
    KMV_CUDA(h, cudaMemsetAsync(B.n_active, 0, sizeof(int32_t), st));
    KMV_CUDA(h, launch_mcg_beta(h->dev, L.n_inst, L.chains, m, B.partial, pre ? pre->prz : nullptr, tol, maxiter,
                                B.cols, B.sys_any, B.n_active, st));
    KMV_CUDA(h, launch_mcg_update_p(h->dev, L.n_items, L.chains, L.n_total, m, B.cols, B.sys_any,
                                    pre ? pre->z : B.r, B.p, st));
  }
  return KMV_OK;
}

// The multi-column solve with the KMV_BF16_HILO operator to FP32 accuracy, by
// the iterative refinement of run_cg_refined applied per column: true residual
// with the FP32 operator, correction by multi-column CG with the tensor-core
// operator, until every column has converged or stagnated.
kmv_status run_mcg_refined(kmv_handle h, const kmv_points* pts, const double* theta, const float* shifts, int m,
                           const float* b, float* x, int warm, double tol, int maxiter, int32_t* col_status,
                           int32_t* col_iters, const McgBufs& B, const McgBufs& R, float* dx, double* prev_rr,
                           cudaStream_t st) {
  const Layout& L = h->layout;
  const int64_t n_cols = (int64_t)L.n_inst * L.chains * m;
  const int64_t nvec = (int64_t)L.chains * L.n_total * m;
  // the relative accuracy of the m-column tensor-core product: the FMA-pipe form
  // with the three-way split for m <= 2, else the two-way split
  const double floor_tol = (m <= 2 && x_width_fma_ok(pts->d)) ? 1e-5 : 1e-3;
  double* worst = reinterpret_cast<double*>(reinterpret_cast<char*>(R.n_active) + 8);
  const int max_outer = 12;
  if (!warm) {
    if (nvec > 0) KMV_CUDA(h, cudaMemsetAsync(x, 0, sizeof(float) * nvec, st));
    KMV_CUDA(h, cudaMemsetAsync(col_status, 0, sizeof(int32_t) * n_cols, st));
    KMV_CUDA(h, cudaMemsetAsync(col_iters, 0, sizeof(int32_t) * n_cols, st));
  }
  KmvArgs a = base_args(h, pts, theta);
  a.m = m;
  a.col_shift = shifts;
  a.col_shift_stride = m;
  for (int outer = 0; outer <= max_outer; ++outer) {
    // r = b - (A + shift) x with the FP32 operator; per-column stopping test
    a.V = x;
    a.Y = R.q;
    KMV_TRY(simt_forward(h, a, st));
    KMV_CUDA(h, launch_mcg_init(h->dev, L.n_items, L.chains, L.n_total, m, b, 0, R.q, 1, x, R.r, R.p, R.partial2,
                                st));
    KMV_CUDA(h, launch_mcg_reduce_init(h->dev, L.n_inst, L.chains, m, R.partial2, tol, R.cols, R.sys_any,
                                       R.n_active, st));
    KMV_CUDA(h, launch_mcg_refine(n_cols, outer, R.cols, prev_rr, R.n_active, worst, st));
    if (outer > 0) KMV_CUDA(h, launch_mcg_undo(h->dev, L.n_items, L.chains, L.n_total, m, R.cols, dx, x, st));
    KMV_CUDA(h, cudaMemcpyAsync(h->host_flag, R.n_active, 16, cudaMemcpyDeviceToHost, st));
    KMV_CUDA(h, cudaStreamSynchronize(st));
    if (*h->host_flag == 0 || outer == max_outer) break;
    double wr;
    std::memcpy(&wr, reinterpret_cast<const char*>(h->host_flag) + 8, sizeof(double));
    const double ratio = wr > 0.0 ? std::sqrt(wr) : 1.0;
    const double inner_tol = std::min(0.5, std::max(floor_tol, 0.5 * tol / ratio));
    // correction of the columns still active (the others get a zero right-hand side)
    KMV_CUDA(h, launch_mcg_mask(h->dev, L.n_items, L.chains, L.n_total, m, R.cols, R.r, st));
    KMV_TRY(run_mcg(h, pts, theta, shifts, m, R.r, 1, dx, inner_tol, maxiter, 0, B, KMV_BF16_HILO, st));
    KMV_CUDA(h, launch_axpy(nvec, dx, x, st));
    KMV_CUDA(h, launch_mcg_finish(n_cols, B.cols, 1, col_status, col_iters, st));
  }
  KMV_CUDA(h, launch_mcg_refine_finish(n_cols, R.cols, col_status, st));
  return KMV_OK;
}

// --- multi-shift CG: all shifts from one Krylov sequence per system ------------------

struct MscgBufs {
  float *r, *p, *q, *ps;
  double* partial;
  MscgSys* sys;
  MscgShift* sh;
  float* base;
  int32_t *sys_active, *n_active;
  uint32_t* count;   // 2 n_sys counters of the fused iteration (alpha step, beta step)
};

void mscg_layout(const Layout& L, int m, Arena& ar, size_t off[10]) {
  const size_t vec = sizeof(float) * (size_t)L.chains * std::max<int64_t>(1, L.n_total);
  const size_t items = (size_t)std::max(1, L.n_items) * L.chains;
  const size_t n_sys = (size_t)L.n_inst * L.chains;
  off[0] = ar.take(vec);
  off[1] = ar.take(vec);
  off[2] = ar.take(vec);
  off[3] = ar.take(vec * m);
  off[4] = ar.take(sizeof(double) * items);
  off[5] = ar.take(sizeof(MscgSys) * n_sys);
  off[6] = ar.take(sizeof(MscgShift) * n_sys * m);
  off[7] = ar.take(sizeof(float) * n_sys);
  off[8] = ar.take(sizeof(int32_t) * n_sys);
  off[9] = ar.take(sizeof(int32_t) * 4 + sizeof(uint32_t) * 2 * n_sys);
}

MscgBufs mscg_bufs(kmv_handle h, const size_t off[10]) {
  MscgBufs b;
  b.r = at<float>(h, off[0]);
  b.p = at<float>(h, off[1]);
  b.q = at<float>(h, off[2]);
  b.ps = at<float>(h, off[3]);
  b.partial = at<double>(h, off[4]);
  b.sys = at<MscgSys>(h, off[5]);
  b.sh = at<MscgShift>(h, off[6]);
  b.base = at<float>(h, off[7]);
  b.sys_active = at<int32_t>(h, off[8]);
  b.n_active = at<int32_t>(h, off[9]);
  b.count = reinterpret_cast<uint32_t*>(b.n_active + 4);
  return b;
}

// (A(theta_s) + shifts[s m + j] I) x_j = b for the m shifts of every system,
// cold start, by multi-shift CG: one m = 1 product with the base (smallest)
// shift per iteration.  x is (chains, N, m); per-shift results go to
// col_status / col_iters (n_sys * m).
kmv_status run_mscg(kmv_handle h, const kmv_points* pts, const double* theta, const float* shifts, int m,
                    const float* b, float* x, double tol, int maxiter, int32_t* col_status, int32_t* col_iters,
                    const MscgBufs& B, kmv_precision prec, cudaStream_t st) {
  const Layout& L = h->layout;
  const int64_t n_cols = (int64_t)L.n_inst * L.chains * m;
  KMV_CUDA(h, launch_mscg_init(h->dev, L.n_items, L.chains, L.n_total, m, b, B.r, B.p, x, B.ps, B.partial, st));
  KMV_CUDA(h, cudaMemsetAsync(B.n_active, 0, sizeof(int32_t), st));
  KMV_CUDA(h, launch_mscg_setup(h->dev, L.n_inst, L.chains, m, B.partial, shifts, tol, B.sys, B.sh, B.base,
                                B.sys_active, B.n_active, st));
  KmvArgs a = base_args(h, pts, theta);
  a.m = 1;
  a.col_shift = B.base;
  a.col_shift_stride = 1;
  a.V = B.p;
  a.Y = B.q;
  a.sys_active = B.sys_active;
  a.dot_partial = B.partial;
  // As in run_cg: the alpha step in the product's epilogue and the beta step
  // in the x, r update (last CTA per system), and with the tensor-core
  // FMA-pipe product the direction updates in its tile preparation.
  const int n_sys = L.n_inst * L.chains;
  const bool tc_fma = prec == KMV_BF16_HILO && x_width_fma_ok(pts->d);
  const bool fused = L.n_items > 0 && (tc_fma || prec == KMV_FP32);
  if (fused) {
    KMV_CUDA(h, cudaMemsetAsync(B.count, 0, sizeof(uint32_t) * 2 * n_sys, st));
    a.ms_sys = B.sys;
    a.ms_sh = B.sh;
    a.ms_m = m;
    a.ms_ps = B.ps;
    a.cg_active = B.sys_active;
    a.cg_n_active = B.n_active;
    a.cg_count = B.count;
    a.cg_r = B.r;
  }
  const int check_every = 4;
  for (int it = 0; it < maxiter; ++it) {
    if (it % check_every == 0) {
      KMV_CUDA(h, cudaMemcpyAsync(h->host_flag, B.n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      KMV_CUDA(h, cudaStreamSynchronize(st));
      if (*h->host_flag == 0) break;
    }
    KMV_TRY(run_forward(h, a, prec, st));
    if (fused) {
      KMV_CUDA(h, launch_mscg_update_xr_beta(h->dev, L.n_items, L.chains, L.n_total, m, B.sys, B.sh, B.sys_active,
                                             B.r, B.q, x, B.ps, B.partial, B.count + n_sys, tol, maxiter, B.n_active,
                                             st));
      if (!tc_fma)
        KMV_CUDA(h, launch_mscg_update_p(h->dev, L.n_items, L.chains, L.n_total, m, B.sys, B.sh, B.sys_active, B.r,
                                         B.p, B.ps, st));
      continue;
    }
    KMV_CUDA(h, launch_mscg_alpha(h->dev, L.n_inst, L.chains, m, B.partial, B.sys, B.sh, B.sys_active, st));
    KMV_CUDA(h, launch_mscg_update_xr(h->dev, L.n_items, L.chains, L.n_total, m, B.sys, B.sh, B.sys_active, B.r,
                                      B.q, x, B.ps, B.partial, st));
    KMV_CUDA(h, cudaMemsetAsync(B.n_active, 0, sizeof(int32_t), st));
    KMV_CUDA(h, launch_mscg_beta(h->dev, L.n_inst, L.chains, m, B.partial, tol, maxiter, B.sys, B.sh, B.sys_active,
                                 B.n_active, st));
    KMV_CUDA(h, launch_mscg_update_p(h->dev, L.n_items, L.chains, L.n_total, m, B.sys, B.sh, B.sys_active, B.r, B.p,
                                     B.ps, st));
  }
  KMV_CUDA(h, launch_mscg_finish(n_cols, B.sh, col_status, col_iters, st));
  return KMV_OK;
}

kmv_status check_prec(kmv_handle h, kmv_precision prec) {
  if (prec != KMV_FP32 && prec != KMV_BF16_HILO) return fail(h, KMV_EINVAL, "unknown precision");
  return KMV_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

kmv_status kmv_create(kmv_handle* out, int device) {
  if (!out) return KMV_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return KMV_ECUDA;
  }
  if (device < 0 || device >= n) return KMV_EINVAL;
  kmv_handle h = new (std::nothrow) kmv_handle_s();
  if (!h) return KMV_ENOMEM;
  h->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&h->host_flag), 64) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    if (h->host_flag) cudaFreeHost(h->host_flag);
    if (h->side) cudaStreamDestroy(h->side);
    delete h;
    return KMV_ECUDA;
  }
  *out = h;
  return KMV_OK;
}

kmv_status kmv_destroy(kmv_handle h) {
  if (!h) return KMV_EINVAL;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  tc_release(h);
  if (h->ws) cudaFree(h->ws);
  if (h->tables) cudaFree(h->tables);
  if (h->cheb_buf) cudaFree(h->cheb_buf);
  if (h->simt_part) cudaFree(h->simt_part);
  if (h->host_flag) cudaFreeHost(h->host_flag);
  if (h->side) cudaStreamDestroy(h->side);
  kmv_profile_enable(h, 0);
  for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
  delete h;
  return KMV_OK;
}

const char* kmv_status_string(kmv_status s) {
  switch (s) {
    case KMV_OK: return "ok";
    case KMV_EINVAL: return "invalid argument";
    case KMV_ENOMEM: return "out of device memory";
    case KMV_ECUDA: return "CUDA error";
    case KMV_ENOTCONV: return "solver did not converge";
    case KMV_ETIMEOUT: return "device-side wait timed out";
    case KMV_ENONFINITE: return "non-finite value";
    case KMV_EUNSUPPORTED: return "unsupported shape or precision";
  }
  return "unknown status";
}

const char* kmv_last_error(kmv_handle h) { return h ? h->last_error.c_str() : ""; }

int64_t kmv_workspace_bytes(kmv_handle h) {
  return h ? (int64_t)(h->ws_bytes + h->tables_bytes + h->cheb_bytes + tc_workspace_bytes(h)) : 0;
}

kmv_status kmv_forward(kmv_handle h, const kmv_points* pts, int32_t chains, const double* theta,
                       const float* V, int32_t m, const float* col_shift, float* Y, double* Y64,
                       kmv_precision prec, void* stream) {
  KMV_TRY(check_points(h, pts, chains));
  KMV_TRY(check_prec(h, prec));
  if (m < 1) return fail(h, KMV_EINVAL, "m must be >= 1");
  if (!theta || !V || !Y) return fail(h, KMV_EINVAL, "theta, V and Y must be non-NULL");
  if ((const void*)V == (const void*)Y) return fail(h, KMV_EINVAL, "Y must not alias V");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KMV_TRY(prepare_layout(h, pts, chains, st));
  KMV_TRY(cheb_prepare(h, pts, theta, 0, st));
  KmvArgs a = base_args(h, pts, theta);
  a.V = V;
  a.m = m;
  a.col_shift = col_shift;
  a.Y = Y;
  a.Y64 = Y64;
  return run_forward(h, a, prec, st);
}

kmv_status kmv_backward(kmv_handle h, const kmv_points* pts, int32_t chains, const double* theta,
                        const float* V, const float* G, int32_t m, double* grad_theta,
                        float* grad_V, kmv_precision prec, void* stream) {
  KMV_TRY(check_points(h, pts, chains));
  KMV_TRY(check_prec(h, prec));
  if (m < 1) return fail(h, KMV_EINVAL, "m must be >= 1");
  if (!theta || !V || !G || !grad_theta) return fail(h, KMV_EINVAL, "theta, V, G, grad_theta must be non-NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KMV_TRY(prepare_layout(h, pts, chains, st));
  Arena ar;
  const size_t o_part = ar.take(backward_ws_bytes(h->layout, m));
  KMV_TRY(reserve(h, ar.used));
  KMV_TRY(cheb_prepare(h, pts, theta, m, st));
  KmvArgs a = base_args(h, pts, theta);
  a.V = V;
  a.G = G;
  a.m = m;
  a.Y = grad_V;
  return run_backward(h, a, grad_theta, at<double>(h, o_part), prec, st);
}

kmv_status kmv_cg_solve(kmv_handle h, const kmv_points* pts, int32_t chains, const double* theta,
                        const float* rhs, int32_t rhs_per_chain, float* x, double tol,
                        int32_t maxiter, int32_t warm_start, int32_t* chain_status, int32_t* iters,
                        kmv_precision prec, void* stream) {
  KMV_TRY(check_points(h, pts, chains));
  KMV_TRY(check_prec(h, prec));
  if (!theta || !rhs || !x || !chain_status) return fail(h, KMV_EINVAL, "NULL argument");
  if (!(tol > 0.0) || maxiter < 1) return fail(h, KMV_EINVAL, "tol must be > 0 and maxiter >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KMV_TRY(prepare_layout(h, pts, chains, st));
  Arena ar;
  SolveLayout SL;
  solve_layout(h, ar, prec, SL);
  KMV_TRY(reserve(h, ar.used));
  KMV_TRY(cheb_prepare(h, pts, theta, 0, st));
  const int64_t stride = rhs_per_chain ? h->layout.n_total : 0;
  return run_solve(h, pts, theta, rhs, stride, x, tol, maxiter, warm_start, chain_status, iters, SL, prec, st);
}

kmv_status kmv_phi_refresh(kmv_handle h, const kmv_points* pts, int32_t chains, const double* theta,
                           const float* xi, float* phi, int32_t n_poles, double cg_tol, int32_t cg_maxiter,
                           int32_t* chain_status, int32_t* cg_iters, double* poles_out, kmv_precision prec,
                           void* stream) {
  KMV_TRY(check_points(h, pts, chains));
  KMV_TRY(check_prec(h, prec));
  if (!theta || !xi || !phi || !chain_status) return fail(h, KMV_EINVAL, "NULL argument");
  if (n_poles < 1 || n_poles > kMaxPoles) return fail(h, KMV_EINVAL, "n_poles must be in [1, 32]");
  if (!(cg_tol > 0.0) || cg_maxiter < 1) return fail(h, KMV_EINVAL, "cg_tol must be > 0 and cg_maxiter >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KMV_TRY(prepare_layout(h, pts, chains, st));
  const Layout& L = h->layout;
  const int n_theta = L.n_theta, n_items = L.n_items;
  const int64_t n_total = L.n_total;
  const int n_sys = L.n_inst * chains;
  const int64_t n_cols = (int64_t)n_sys * n_poles;
  // the multi-shift solve's product is single-column: FP32-accurate in both
  // forms where the three-way split fits, else the BF16 form polishes by refinement
  const bool refined = prec == KMV_BF16_HILO && !x_width_fma_ok(L.d);
  // with a preconditioner set (and matching this layout) the shifted systems run
  // as preconditioned columns of one multi-column CG (a preconditioner breaks the
  // shift invariance multi-shift CG relies on); without, multi-shift CG
  const bool use_pc = h->pc_on && h->pc.n_inst == L.n_inst && h->pc.chains == L.chains &&
                      h->pc.n_total == L.n_total;
  if (h->pc_on && !use_pc)
    return fail(h, KMV_EINVAL, "the preconditioner was built for another layout (n_inst, chains, N_total)");
  Arena ar;
  size_t ob[8], orf[8], oms[10], opre[4];
  if (!use_pc) mscg_layout(L, n_poles, ar, oms);
  if (refined || use_pc) mcg_layout(L, n_poles, ar, ob);
  if (refined && !use_pc) mcg_layout(L, n_poles, ar, orf);
  if (use_pc) mcg_pre_layout(L, n_poles, h->pc.rank, ar, opre);
  const size_t vec1 = sizeof(float) * (size_t)chains * std::max<int64_t>(1, n_total);
  const size_t o_x = ar.take(sizeof(float) * (size_t)chains * std::max<int64_t>(1, n_total) * n_poles);
  const size_t o_sh = ar.take(sizeof(float) * (size_t)n_cols);
  const size_t o_w = ar.take(sizeof(double) * (size_t)n_cols);
  const size_t o_bnd = ar.take(sizeof(double) * (size_t)n_sys);
  const size_t o_cst = ar.take(sizeof(int32_t) * (size_t)n_cols), o_cit = ar.take(sizeof(int32_t) * (size_t)n_cols);
  const size_t o_prev = ar.take(sizeof(double) * (size_t)n_cols);
  const size_t o_dx = refined ? ar.take(sizeof(float) * (size_t)chains * std::max<int64_t>(1, n_total) * n_poles) : 0;
  const size_t o_one = ar.take(vec1), o_y = ar.take(vec1);
  KMV_TRY(reserve(h, ar.used));
  char* base = static_cast<char*>(h->ws);
  float* x_p = reinterpret_cast<float*>(base + o_x);
  float* shifts = reinterpret_cast<float*>(base + o_sh);
  double* weights = reinterpret_cast<double*>(base + o_w);
  double* bounds = reinterpret_cast<double*>(base + o_bnd);
  int32_t* col_status = reinterpret_cast<int32_t*>(base + o_cst);
  int32_t* col_iters = reinterpret_cast<int32_t*>(base + o_cit);
  double* prev_rr = reinterpret_cast<double*>(base + o_prev);
  float* dx = refined ? reinterpret_cast<float*>(base + o_dx) : nullptr;
  float* ones = reinterpret_cast<float*>(base + o_one);
  float* y1 = reinterpret_cast<float*>(base + o_y);
  KMV_TRY(cheb_prepare(h, pts, theta, 0, st));

  // spectral interval [sigma^2, max row sum of A] from A 1 (App. A, read with the
  // exact row-sum bound); 1% slack covers the rounding of the product
  KMV_CUDA(h, launch_phi_fill(ones, (int64_t)chains * n_total, 1.0f, st));
  {
    KmvArgs a = base_args(h, pts, theta);
    a.m = 1;
    a.V = ones;
    a.Y = y1;
    KMV_TRY(run_forward(h, a, prec, st));
  }
  KMV_CUDA(h, launch_phi_bounds(h->dev, n_sys, chains, n_total, y1, 1.01, bounds, st));
  KMV_CUDA(h, launch_phi_poles(n_sys, n_theta, n_poles, theta, bounds, shifts, weights, poles_out, st));
  if (use_pc) {
    // FP32 products in both forms: the n_poles-column tensor-core product (1e-3)
    // is too coarse to refine the small-shift systems when sigma^2 is small next
    // to |K|, and with the preconditioner the solve takes few iterations
    const McgPre pre = mcg_pre(h, opre);
    const McgBufs B = mcg_bufs(h, ob);
    KMV_TRY(run_mcg(h, pts, theta, shifts, n_poles, xi, 0, x_p, cg_tol, cg_maxiter, 0, B, KMV_FP32, st, &pre));
    KMV_CUDA(h, launch_mcg_finish(n_cols, B.cols, 0, col_status, col_iters, st));
  } else {
    // the n_poles shifted systems of every (instance, chain) from one Krylov sequence
    KMV_TRY(run_mscg(h, pts, theta, shifts, n_poles, xi, x_p, cg_tol, cg_maxiter, col_status, col_iters,
                     mscg_bufs(h, oms), prec, st));
    if (refined) {
      // the BF16 operator leaves the shifted solves at its own accuracy: polish each
      // to cg_tol by refinement with FP32 residuals (a check only, where they are there)
      KMV_TRY(run_mcg_refined(h, pts, theta, shifts, n_poles, xi, x_p, 1, cg_tol, cg_maxiter, col_status,
                              col_iters, mcg_bufs(h, ob), mcg_bufs(h, orf), dx, prev_rr, st));
    }
  }
  KMV_CUDA(h, launch_phi_combine(h->dev, n_items, chains, n_poles, n_total, weights, x_p, phi, st));
  KMV_CUDA(h, launch_phi_status(n_sys, n_poles, col_status, col_iters, chain_status, cg_iters, st));
  return KMV_OK;
}

kmv_status kmv_nystrom_build(kmv_handle h, const kmv_points* pts, int32_t chains, const double* theta,
                             int32_t rank, const float* omega, float* U, double* lam, int32_t* chain_status,
                             kmv_precision prec, void* stream) {
  KMV_TRY(check_points(h, pts, chains));
  KMV_TRY(check_prec(h, prec));
  if (!theta || !omega || !U || !lam || !chain_status) return fail(h, KMV_EINVAL, "NULL argument");
  if (rank < 1 || rank > kMaxRank) return fail(h, KMV_EINVAL, "rank must be in [1, 128]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KMV_TRY(prepare_layout(h, pts, chains, st));
  if (h->capturing) return fail(h, KMV_EINVAL, "kmv_nystrom_build cannot run during stream capture");
  const Layout& L = h->layout;
  const size_t n_sys = (size_t)L.n_inst * L.chains;
  const size_t rr = (size_t)rank * rank;
  Arena ar;
  const size_t o_y = ar.take(sizeof(float) * (size_t)L.chains * std::max<int64_t>(1, L.n_total) * rank);
  const size_t o_g = ar.take(sizeof(double) * n_sys * 3 * rr);
  const size_t o_s = ar.take(sizeof(double) * n_sys * 4 * rr);
  const size_t o_t = ar.take(sizeof(double) * n_sys * rr);
  const size_t o_nu = ar.take(sizeof(double) * n_sys);
  KMV_TRY(reserve(h, ar.used));
  KMV_TRY(cheb_prepare(h, pts, theta, 0, st));
  // Y = K Omega: the product without the noise term
  KmvArgs a = base_args(h, pts, theta);
  a.V = omega;
  a.m = rank;
  a.Y = at<float>(h, o_y);
  a.no_diag = 1;
  KMV_TRY(run_forward(h, a, prec, st));
  KMV_CUDA(h, launch_nystrom_finish(h->dev, L.n_items, L.n_inst, L.chains, L.n_total, rank, omega, at<float>(h, o_y),
                                    at<double>(h, o_g), at<double>(h, o_s), at<double>(h, o_t), at<double>(h, o_nu), U,
                                    lam, chain_status, st));
  return KMV_OK;
}

kmv_status kmv_set_preconditioner(kmv_handle h, const kmv_nystrom* pc) {
  if (!h) return KMV_EINVAL;
  if (!pc) {
    h->pc_on = false;
    h->pc = kmv_nystrom{};
    return KMV_OK;
  }
  if (pc->rank < 1 || pc->rank > kMaxRank || !pc->U || !pc->lam || pc->n_inst < 1 || pc->chains < 1 ||
      pc->n_total < 0)
    return fail(h, KMV_EINVAL, "bad preconditioner (rank in [1, 128], U and lam non-NULL, sizes)");
  h->pc = *pc;
  h->pc_on = true;
  return KMV_OK;
}

kmv_status leapfrog_step(kmv_handle h, const kmv_points* pts, int32_t chains, const float* y,
                         const float* phi, double* theta, double* pi, double dt,
                         const double* prior_mu, const double* prior_prec, const uint8_t* free_mask,
                         double cg_tol, int32_t cg_maxiter, float* x_work, int32_t* chain_status,
                         int32_t* cg_iters, kmv_precision prec, void* stream) {
  KMV_TRY(check_points(h, pts, chains));
  KMV_TRY(check_prec(h, prec));
  if (!y || !phi || !theta || !pi || !x_work || !chain_status) return fail(h, KMV_EINVAL, "NULL argument");
  if ((prior_mu == nullptr) != (prior_prec == nullptr))
    return fail(h, KMV_EINVAL, "prior_mu and prior_prec must both be set or both be NULL");
  if (!std::isfinite(dt) || !(cg_tol > 0.0) || cg_maxiter < 1) return fail(h, KMV_EINVAL, "bad dt / cg_tol / cg_maxiter");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KMV_TRY(prepare_layout(h, pts, chains, st));
  const Layout& L = h->layout;
  const int n_sys = L.n_inst * L.chains;
  Arena ar;
  SolveLayout SL;
  solve_layout(h, ar, prec, SL);
  const size_t o_th = ar.take(sizeof(double) * n_sys * L.n_theta);
  const size_t o_gr = ar.take(sizeof(double) * n_sys * L.n_theta);
  const size_t vec2 = sizeof(float) * 2 * (size_t)L.chains * std::max<int64_t>(1, L.n_total);
  const size_t o_vf = ar.take(vec2);
  const size_t o_gf = ar.take(vec2);
  const size_t o_bp = ar.take(backward_ws_bytes(L, 2));
  KMV_TRY(reserve(h, ar.used));
  double* theta_h = at<double>(h, o_th);
  double* grad = at<double>(h, o_gr);
  float* Vf = at<float>(h, o_vf);
  float* Gf = at<float>(h, o_gf);

  // drift: theta_h = theta + dt/2 pi
  KMV_CUDA(h, launch_lf_drift(n_sys, L.n_theta, theta, pi, free_mask, 0.5 * dt, theta_h, st));
  KMV_TRY(cheb_prepare(h, pts, theta_h, 2, st));
  // x = A(theta_h)^{-1} y, cold start (keeps the force a function of theta_h only)
  KMV_TRY(run_solve(h, pts, theta_h, y, 0, x_work, cg_tol, cg_maxiter, 0, chain_status, cg_iters, SL, prec, st));
  // force: d/dtheta [-x^T A x / 2 + phi^T A phi / 2] at frozen x (Eq. u)
  KMV_CUDA(h, launch_pack_force(L.chains, L.n_total, x_work, phi, Vf, Gf, st));
  KmvArgs a = base_args(h, pts, theta_h);
  a.V = Vf;
  a.G = Gf;
  a.m = 2;
  a.Y = nullptr;
  // The two quadratic forms cancel to a small fraction of their size; both
  // adjoint forms keep every pair's term to about FP32 accuracy (the
  // tensor-core form from its split operands and exact Q = Qh + Ql), so the
  // force follows the call's precision.
  KMV_TRY(run_backward(h, a, grad, at<double>(h, o_bp), prec, st));
  // kick + drift
  KMV_CUDA(h, launch_lf_kick_drift(n_sys, L.n_theta, theta_h, grad, prior_mu, prior_prec, free_mask,
                                   chain_status, dt, theta, pi, st));
  return KMV_OK;
}

kmv_status kmv_implicit_step(kmv_handle h, const kmv_points* pts, int32_t chains, const float* y, const float* phi,
                             double* theta, double* pi, double dt, const double* prior_mu, const double* prior_prec,
                             const uint8_t* free_mask, int32_t aa_depth, double tol, int32_t maxiter, float* x_work,
                             int32_t* chain_status, int32_t* iters, kmv_precision prec, void* stream) {
  KMV_TRY(check_points(h, pts, chains));
  KMV_TRY(check_prec(h, prec));
  if (!y || !phi || !theta || !pi || !x_work || !chain_status || !iters)
    return fail(h, KMV_EINVAL, "NULL argument");
  if ((prior_mu == nullptr) != (prior_prec == nullptr))
    return fail(h, KMV_EINVAL, "prior_mu and prior_prec must both be set or both be NULL");
  if (!std::isfinite(dt) || !(tol > 0.0) || maxiter < 1 || aa_depth < 1 || aa_depth > kMaxAA)
    return fail(h, KMV_EINVAL, "bad dt / tol / maxiter, or aa_depth outside [1, 16]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KMV_TRY(prepare_layout(h, pts, chains, st));
  const Layout& L = h->layout;
  if (h->pc_on && (h->pc.n_inst != L.n_inst || h->pc.chains != L.chains || h->pc.n_total != L.n_total))
    return fail(h, KMV_EINVAL, "the preconditioner was built for another layout (n_inst, chains, N_total)");
  const int n_sys = L.n_inst * L.chains, n = L.n_theta, k = aa_depth;
  const size_t vec = (size_t)L.chains * std::max<int64_t>(1, L.n_total);
  const size_t items = (size_t)std::max(1, L.n_items) * L.chains;
  const int rank = h->pc_on ? h->pc.rank : 1;
  Arena ar;
  const size_t o_th0 = ar.take(sizeof(double) * n_sys * n), o_pi0 = ar.take(sizeof(double) * n_sys * n);
  const size_t o_tb = ar.take(sizeof(double) * n_sys * n), o_gr = ar.take(sizeof(double) * n_sys * n);
  const size_t o_vf = ar.take(sizeof(float) * 2 * vec), o_gf = ar.take(sizeof(float) * 2 * vec);
  const size_t o_bp = ar.take(backward_ws_bytes(L, 2));
  const size_t o_q = ar.take(sizeof(float) * vec), o_r = ar.take(sizeof(float) * vec), o_z = ar.take(sizeof(float) * vec);
  const size_t o_gx = ar.take(sizeof(float) * vec * k), o_fx = ar.take(sizeof(float) * vec * k);
  const size_t o_gtp = ar.take(sizeof(double) * (size_t)k * n_sys * 2 * n);
  const size_t o_ftp = ar.take(sizeof(double) * (size_t)k * n_sys * 2 * n);
  const size_t o_h = ar.take(sizeof(double) * (size_t)n_sys * k * k), o_al = ar.take(sizeof(double) * (size_t)n_sys * k);
  const size_t o_act = ar.take(sizeof(int32_t) * n_sys), o_dn = ar.take(sizeof(int32_t) * n_sys);
  const size_t o_na = ar.take(sizeof(int32_t) * 4);
  const size_t o_xp = ar.take(sizeof(double) * items * k), o_rp = ar.take(sizeof(double) * items * 2);
  const size_t o_c = ar.take(sizeof(double) * n_sys), o_pp = ar.take(sizeof(double) * items);
  const size_t o_proj = ar.take(sizeof(double) * items * rank), o_coef = ar.take(sizeof(double) * n_sys * rank);
  const size_t o_prz = ar.take(sizeof(double) * items);
  const size_t o_brr = ar.take(sizeof(double) * n_sys), o_bit = ar.take(sizeof(int32_t) * n_sys);
  KMV_TRY(reserve(h, ar.used));
  double* th0 = at<double>(h, o_th0);
  double* pi0 = at<double>(h, o_pi0);
  double* tb = at<double>(h, o_tb);
  double* grad = at<double>(h, o_gr);
  float* q = at<float>(h, o_q);
  float* r = at<float>(h, o_r);
  float* z = at<float>(h, o_z);
  int32_t* active = at<int32_t>(h, o_act);
  int32_t* n_active = at<int32_t>(h, o_na);
  double* cscale = at<double>(h, o_c);
  const PcgPrecond P{h->pc.rank, h->pc.U, h->pc.lam};
  KMV_CUDA(h, cudaMemcpyAsync(th0, theta, sizeof(double) * n_sys * n, cudaMemcpyDeviceToDevice, st));
  KMV_CUDA(h, cudaMemcpyAsync(pi0, pi, sizeof(double) * n_sys * n, cudaMemcpyDeviceToDevice, st));

  // c ~ rho(R~ A(theta_0)) by 20 power iterations from the vector of ones, times 1.05
  KMV_TRY(cheb_prepare(h, pts, th0, 2, st));
  {
    KmvArgs a = base_args(h, pts, th0);
    a.m = 1;
    KMV_CUDA(h, launch_phi_fill(z, (int64_t)vec, 1.0f, st));
    KMV_CUDA(h, launch_imp_scale(h->dev, L.n_items, L.chains, L.n_total, nullptr, z, z, at<double>(h, o_pp), st));
    KMV_CUDA(h, launch_imp_norm(h->dev, L.n_inst, L.chains, at<double>(h, o_pp), cscale, st));
    KMV_CUDA(h, launch_imp_scale(h->dev, L.n_items, L.chains, L.n_total, cscale, z, r, at<double>(h, o_pp), st));
    for (int t = 0; t < 20; ++t) {
      a.V = r;
      a.Y = q;
      KMV_TRY(run_forward(h, a, KMV_FP32, st));
      const float* w = q;
      if (h->pc_on) {
        KMV_CUDA(h, launch_pcg_precond(h->dev, L.n_items, L.n_inst, L.chains, L.n_total, P, th0, n, q, z, nullptr,
                                       at<double>(h, o_proj), at<double>(h, o_coef), at<double>(h, o_prz), st));
        w = z;
      }
      KMV_CUDA(h, launch_imp_scale(h->dev, L.n_items, L.chains, L.n_total, nullptr, w, z, at<double>(h, o_pp), st));
      KMV_CUDA(h, launch_imp_norm(h->dev, L.n_inst, L.chains, at<double>(h, o_pp), cscale, st));
      KMV_CUDA(h, launch_imp_scale(h->dev, L.n_items, L.chains, L.n_total, cscale, z, r, at<double>(h, o_pp), st));
    }
    KMV_CUDA(h, launch_imp_cfinal(n_sys, 1.05, cscale, st));
  }

  // Anderson-accelerated iteration of Phi, all systems in lockstep, finished ones masked
  KMV_CUDA(h, launch_fill_i32(active, n_sys, 1, st));
  KMV_CUDA(h, cudaMemsetAsync(chain_status, 0, sizeof(int32_t) * n_sys, st));
  KMV_CUDA(h, cudaMemsetAsync(iters, 0, sizeof(int32_t) * n_sys, st));
  // Phi's linear part takes the FP32 product in both forms: Anderson acceleration
  // measures the true residual y - A x each iteration, and on ill-conditioned
  // systems the tensor-core product's rounding kept it above tol (measured: a
  // kappa ~ 1.5e3 system stalled for 1500 iterations that FP32 solves in 270);
  // the adjoint of the force, FP32 as well, is most of an iteration's cost
  const kmv_precision lin_prec = KMV_FP32;
  (void)prec;
  const int check_every = 4;
  for (int it = 0; it < maxiter; ++it) {
    if (!h->capturing && it > 0 && it % check_every == 0) {
      KMV_CUDA(h, cudaMemcpyAsync(h->host_flag, n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      KMV_CUDA(h, cudaStreamSynchronize(st));
      if (*h->host_flag == 0) break;
    }
    const int slot = it % k, cnt = std::min(it + 1, k);
    KMV_CUDA(h, launch_imp_mid(n_sys * n, th0, theta, tb, st));
    KMV_TRY(cheb_prepare(h, pts, tb, 2, st));
    KmvArgs a = base_args(h, pts, tb);
    a.m = 1;
    a.V = x_work;
    a.Y = q;
    a.sys_active = active;
    KMV_TRY(run_forward(h, a, lin_prec, st));
    KMV_CUDA(h, launch_imp_resid(h->dev, L.n_items, L.chains, L.n_total, y, q, active, r, at<double>(h, o_rp), st));
    const float* zz = r;
    if (h->pc_on) {
      KMV_CUDA(h, launch_pcg_precond(h->dev, L.n_items, L.n_inst, L.chains, L.n_total, P, th0, n, r, z, active,
                                     at<double>(h, o_proj), at<double>(h, o_coef), at<double>(h, o_prz), st));
      zz = z;
    }
    KMV_CUDA(h, launch_imp_x(h->dev, L.n_items, L.chains, L.n_total, k, slot, cnt, x_work, zz, cscale, active,
                             at<float>(h, o_gx), at<float>(h, o_fx), at<double>(h, o_xp), st));
    // the frozen-x force at theta_bar (FP32 adjoint, as in the leapfrog step)
    KMV_CUDA(h, launch_pack_force(L.chains, L.n_total, x_work, phi, at<float>(h, o_vf), at<float>(h, o_gf), st));
    KmvArgs fa = base_args(h, pts, tb);
    fa.V = at<float>(h, o_vf);
    fa.G = at<float>(h, o_gf);
    fa.m = 2;
    fa.Y = nullptr;
    fa.sys_active = active;
    KMV_TRY(run_backward(h, fa, grad, at<double>(h, o_bp), KMV_FP32, st));
    KMV_CUDA(h, cudaMemsetAsync(n_active, 0, sizeof(int32_t), st));
    KMV_CUDA(h, launch_imp_aa(h->dev, L.n_inst, L.chains, n, k, slot, cnt, th0, pi0, theta, pi, grad, prior_mu,
                              prior_prec, free_mask, dt, at<double>(h, o_xp), at<double>(h, o_rp), tol, it, maxiter,
                              at<double>(h, o_gtp), at<double>(h, o_ftp), at<double>(h, o_h), at<double>(h, o_al),
                              active, at<int32_t>(h, o_dn), chain_status, iters, n_active, at<double>(h, o_brr),
                              at<int32_t>(h, o_bit), st));
    KMV_CUDA(h, launch_imp_mix(h->dev, L.n_items, L.n_inst, L.chains, L.n_total, n, k, slot, cnt,
                               at<double>(h, o_gtp), at<float>(h, o_gx), at<double>(h, o_al), active,
                               at<int32_t>(h, o_dn), theta, pi, x_work, st));
  }
  return KMV_OK;
}

kmv_status kmv_status_merge(int32_t n, const int32_t* src, int32_t* dst, void* stream) {
  if (n < 0 || (n > 0 && (!src || !dst))) return KMV_EINVAL;
  return launch_status_merge(n, src, dst, static_cast<cudaStream_t>(stream)) == cudaSuccess ? KMV_OK : KMV_ECUDA;
}

kmv_status kmv_accept(int32_t n_sys, int32_t n_theta, const double* H_old, const double* H_new, const double* u,
                      const int32_t* status, const double* theta_old, double* theta, int32_t* accepted,
                      void* stream) {
  if (n_sys < 0 || n_theta < 1) return KMV_EINVAL;
  if (n_sys > 0 && (!H_old || !H_new || !u || !theta_old || !theta || !accepted)) return KMV_EINVAL;
  return launch_accept(n_sys, n_theta, H_old, H_new, u, status, theta_old, theta, accepted,
                       static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? KMV_OK
             : KMV_ECUDA;
}

kmv_status kmv_energy(kmv_handle h, const kmv_points* pts, int32_t chains, const float* y,
                      const float* phi, const double* theta, const double* pi,
                      const double* prior_mu, const double* prior_prec, double cg_tol,
                      int32_t cg_maxiter, float* x_work, double* H, double* terms,
                      int32_t* chain_status, int32_t* cg_iters, kmv_precision prec, void* stream) {
  KMV_TRY(check_points(h, pts, chains));
  KMV_TRY(check_prec(h, prec));
  if (!y || !phi || !theta || !x_work || !H || !chain_status) return fail(h, KMV_EINVAL, "NULL argument");
  if ((prior_mu == nullptr) != (prior_prec == nullptr))
    return fail(h, KMV_EINVAL, "prior_mu and prior_prec must both be set or both be NULL");
  if (!(cg_tol > 0.0) || cg_maxiter < 1) return fail(h, KMV_EINVAL, "bad cg_tol / cg_maxiter");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KMV_TRY(prepare_layout(h, pts, chains, st));
  const Layout& L = h->layout;
  Arena ar;
  SolveLayout SL;
  solve_layout(h, ar, prec, SL);
  const size_t vec = (size_t)L.chains * std::max<int64_t>(1, L.n_total);
  const size_t o_y = ar.take(sizeof(float) * vec);
  const size_t o_y64 = ar.take(sizeof(double) * vec);
  const size_t items = (size_t)std::max(1, L.n_items) * L.chains;
  const size_t o_p1 = ar.take(sizeof(double) * items);
  const size_t o_p2 = ar.take(sizeof(double) * items);
  KMV_TRY(reserve(h, ar.used));
  KMV_TRY(cheb_prepare(h, pts, theta, 0, st));
  KMV_TRY(run_solve(h, pts, theta, y, 0, x_work, cg_tol, cg_maxiter, 0, chain_status, cg_iters, SL, prec, st));
  KmvArgs a = base_args(h, pts, theta);
  a.V = phi;
  a.m = 1;
  a.Y = at<float>(h, o_y);
  a.Y64 = at<double>(h, o_y64);
  KMV_TRY(run_forward(h, a, prec, st));
  if (L.n_items > 0) {
    KMV_CUDA(h, launch_dot_partial(h->dev, L.n_items, L.chains, L.n_total, y, 0, x_work, nullptr,
                                   at<double>(h, o_p1), st));
    KMV_CUDA(h, launch_dot_partial(h->dev, L.n_items, L.chains, L.n_total, phi, L.n_total, nullptr,
                                   at<double>(h, o_y64), at<double>(h, o_p2), st));
  }
  KMV_CUDA(h, launch_energy_finalize(h->dev, L.n_inst, L.chains, L.n_theta, theta, pi, prior_mu,
                                     prior_prec, at<double>(h, o_p1), at<double>(h, o_p2),
                                     chain_status, H, terms, st));
  return KMV_OK;
}

}  // extern "C"
