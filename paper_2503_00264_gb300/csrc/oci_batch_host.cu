// oci_batch_host.cu -- host side of the batched form: setup (class packing,
// per-slab type tables, per-class autotuned tile size), the per-time-step graph
// and the batch entry points of the C ABI.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "oci_batch.h"

namespace oci {

#define BCK(call)                                        \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

constexpr int kPad = 128;     // slab padding (multiple of every tile size and of the 32-cell carry block)
constexpr int kMinTile = 8;  // smallest tile (cells) of any sweep candidate
// refinement schedule of the mixed form (as the single-slab FP32 form): refine
// after k_max inner sweeps or once e fell below theta of the block's first;
// OCI_MX_KMAX / OCI_MX_THETA override
constexpr int kBatchMxKmax = 64;
constexpr double kBatchMxTheta = 1e-3;

// [J][K] host/device rows -> class SoA column block: dst[k*stride + j], j < J only.
__global__ void k_bt_in(int J, int stride, int K, const double *__restrict__ src, double *__restrict__ dst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (j < J) dst[(size_t)k * stride + j] = src[(size_t)j * K + k];
}
__global__ void k_bt_out(int J, int stride, int K, const double *__restrict__ src, double *__restrict__ dst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (j < J) dst[(size_t)j * K + k] = src[(size_t)k * stride + j];
}

template <class T>
static int balloc(BatchClass &c, T **p, size_t count, cudaStream_t st) {
  BCK(cudaMalloc(p, count * sizeof(T) + 16));
  BCK(cudaMemsetAsync(*p, 0, count * sizeof(T) + 16, st));
  c.allocs.push_back((void *)*p);
  return OCI_OK;
}
template <class T>
static int bupload(BatchClass &c, T **p, const std::vector<T> &v, cudaStream_t st) {
  int rc = balloc(c, p, v.size(), st);
  if (rc) return rc;
  if (!v.empty()) BCK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return OCI_OK;
}

// tile arrays for tile size cb (tiles never straddle slabs)
static int build_tiles(BatchClass &c, int np, int cb, int32_t *tile_slab, int32_t *tile_first, int32_t *t0,
                       int32_t *t1, cudaStream_t st) {
  std::vector<int32_t> ts, tf, a, b;
  for (size_t i = 0; i < c.h_J.size(); i++) {
    a.push_back((int32_t)ts.size());
    for (int j0 = 0; j0 < c.h_J[i]; j0 += cb) {
      ts.push_back((int32_t)i);
      tf.push_back(c.h_start[i] + j0);
    }
    b.push_back((int32_t)ts.size());
  }
  c.d.n_tiles = (int)ts.size();
  BCK(cudaMemcpyAsync(tile_slab, ts.data(), ts.size() * 4, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(tile_first, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(t0, a.data(), a.size() * 4, cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(t1, b.data(), b.size() * 4, cudaMemcpyHostToDevice, st));
  BCK(cudaStreamSynchronize(st));  // host vectors go out of scope
  c.cb = cb;
  c.np = np;
  const int maxg = np ? b_reg_max_grid(c.d.N, c.d.G, cb, np, c.mixed)
                      : (c.mixed ? b_mx_max_grid(c.d.N, c.d.G, cb) : b_max_grid(c.d.N, c.d.G, cb));
  c.grid = std::min(c.d.n_tiles, maxg);
  if (c.grid < 1) c.grid = 1;
  return OCI_OK;
}

static int setup_class(Batch &B, BatchClass &c, const oci_problem *probs) {
  cudaStream_t st = B.stream;
  const int N = B.N[c.slabs[0]], G = B.G[c.slabs[0]];
  c.d.N = N;
  c.d.G = G;
  c.d.n_slabs = (int)c.slabs.size();
  std::vector<double> mu, w;
  gauss_legendre(N, mu, w);
  std::vector<double> Linv, Cin, Mp, Kap, tdx, tsig, tah, incv, Lcov;
  std::vector<int32_t> type, seg;
  int offset = 0, T = 0;
  for (size_t i = 0; i < c.slabs.size(); i++) {
    const oci_problem &p = probs[c.slabs[i]];
    Handle tmp;
    tmp.J = p.J;
    tmp.N = N;
    tmp.G = G;
    tmp.dt = p.dt;
    tmp.h_dx.assign(p.dx, p.dx + p.J);
    tmp.h_mat.assign(p.mat, p.mat + p.J);
    tmp.h_sigma_t.assign(p.sigma_t, p.sigma_t + (size_t)p.n_mat * G);
    tmp.h_sigma_s.assign(p.sigma_s, p.sigma_s + (size_t)p.n_mat * G * G);
    tmp.h_v.assign(p.v, p.v + G);
    tmp.h_mu = mu;
    tmp.h_w = w;
    std::vector<double> L, C, M, K, dx, sg, Lco;
    int rc = build_tables(tmp, L, C, M, K, dx, sg, Lco);
    if (rc) return rc;
    const int Ts = tmp.tt.n_types;
    Linv.insert(Linv.end(), L.begin(), L.end());
    Cin.insert(Cin.end(), C.begin(), C.end());
    Mp.insert(Mp.end(), M.begin(), M.end());
    Kap.insert(Kap.end(), K.begin(), K.end());
    tdx.insert(tdx.end(), dx.begin(), dx.end());
    tsig.insert(tsig.end(), sg.begin(), sg.end());
    Lcov.insert(Lcov.end(), Lco.begin(), Lco.end());
    for (int t = 0; t < Ts; t++)
      for (int g = 0; g < G; g++) tah.push_back(dx[t] / (2.0 * p.v[g] * p.dt));
    const int Jpad = (p.J + kPad - 1) / kPad * kPad;
    c.h_start.push_back(offset);
    c.h_J.push_back(p.J);
    type.resize(offset + Jpad, 0);
    seg.resize(offset + Jpad, -1);
    for (int j = 0; j < p.J; j++) {
      type[offset + j] = T + tmp.h_type[j];
      seg[offset + j] = (int32_t)i;
    }
    for (int side = 0; side < 2; side++) {
      const double *src = side == 0 ? p.inc_left : p.inc_right;
      for (int k = 0; k < G * N * 2; k++) incv.push_back(src ? src[k] : 0.0);
    }
    offset += Jpad;
    T += Ts;
  }
  const int Jc = offset;
  c.d.Jc = Jc;
  int rc;
  int32_t *d_type, *d_seg, *d_start, *d_J, *d_t0, *d_t1, *d_ts, *d_tf;
  double *d_Linv, *d_Cin, *d_Mp, *d_Kap, *d_tdx, *d_tsig, *d_tah, *d_w, *d_mu, *d_inc;
  if ((rc = bupload(c, &d_type, type, st)) || (rc = bupload(c, &d_seg, seg, st))) return rc;
  std::vector<int32_t> hs(c.h_start.begin(), c.h_start.end()), hj(c.h_J.begin(), c.h_J.end());
  if ((rc = bupload(c, &d_start, hs, st)) || (rc = bupload(c, &d_J, hj, st))) return rc;
  if ((rc = bupload(c, &d_Linv, Linv, st)) || (rc = bupload(c, &d_Cin, Cin, st)) || (rc = bupload(c, &d_Mp, Mp, st)) ||
      (rc = bupload(c, &d_Kap, Kap, st)) || (rc = bupload(c, &d_tdx, tdx, st)) || (rc = bupload(c, &d_tsig, tsig, st)) ||
      (rc = bupload(c, &d_tah, tah, st)) || (rc = bupload(c, &d_w, w, st)) || (rc = bupload(c, &d_mu, mu, st)) ||
      (rc = bupload(c, &d_inc, incv, st)))
    return rc;
  const int max_tiles = Jc / kMinTile + (int)c.slabs.size();
  if ((rc = balloc(c, &d_t0, c.slabs.size(), st)) || (rc = balloc(c, &d_t1, c.slabs.size(), st)) ||
      (rc = balloc(c, &d_ts, max_tiles, st)) || (rc = balloc(c, &d_tf, max_tiles, st)))
    return rc;
  const size_t nPsi = (size_t)G * N * 4 * Jc;
  double *Psi0, *Psi1, *tc, *pp, *phi, *parts, *bparts, *bal, *Q = nullptr;
  if ((rc = balloc(c, &Psi0, nPsi, st)) || (rc = balloc(c, &Psi1, nPsi, st)) || (rc = balloc(c, &tc, nPsi, st)) ||
      (rc = balloc(c, &pp, (size_t)G * N * 2 * Jc, st)) || (rc = balloc(c, &phi, (size_t)G * 4 * Jc, st)) ||
      (rc = balloc(c, &parts, max_tiles, st)) || (rc = balloc(c, &bparts, (size_t)(Jc / 32) * G * 8, st)) ||
      (rc = balloc(c, &bal, (size_t)c.slabs.size() * G * 10, st)))
    return rc;
  bool anyQ = false;
  for (int s : c.slabs) anyQ |= probs[s].Q != nullptr;
  if (anyQ && (rc = balloc(c, &Q, (size_t)G * 4 * Jc, st))) return rc;
  for (size_t i = 0; i < c.slabs.size(); i++) {
    const oci_problem &p = probs[c.slabs[i]];
    if (p.Q) {
      BCK(cudaMemcpyAsync(B.stage, p.Q, (size_t)p.J * G * 4 * 8, cudaMemcpyHostToDevice, st));
      k_bt_in<<<dim3((p.J + 255) / 256, G * 4), 256, 0, st>>>(p.J, Jc, G * 4, B.stage, Q + c.h_start[i]);
    }
    if (p.psi_init) {
      BCK(cudaMemcpyAsync(B.stage, p.psi_init, (size_t)p.J * G * N * 2 * 8, cudaMemcpyHostToDevice, st));
      k_bt_in<<<dim3((p.J + 255) / 256, G * N * 2), 256, 0, st>>>(p.J, Jc, G * N * 2, B.stage, pp + c.h_start[i]);
    }
    BCK(cudaStreamSynchronize(st));
  }
  BatchClassDev &d = c.d;
  d.type = d_type; d.seg = d_seg; d.slab_start = d_start; d.slab_J = d_J; d.slab_tile0 = d_t0; d.slab_tile1 = d_t1;
  d.tile_slab = d_ts; d.tile_first_cell = d_tf;
  d.Linv = d_Linv; d.Cin = d_Cin; d.Mp = d_Mp; d.Kap = d_Kap; d.tdx = d_tdx; d.tsig = d_tsig; d.tah = d_tah;
  d.w = d_w; d.mu = d_mu; d.inc = d_inc; d.Q = Q;
  d.Psi0 = Psi0; d.Psi1 = Psi1; d.tc = tc; d.psi_prev = pp; d.phi = phi; d.partials = parts;
  d.bal_partials = bparts; d.bal = bal;
  if (c.mixed) {
    // FP32 copies of the cell tables, FP32 correction ping-pong and z = Linv r
    auto to32 = [](const std::vector<double> &a) {
      std::vector<float> f(a.size());
      for (size_t i = 0; i < a.size(); i++) f[i] = (float)a[i];
      return f;
    };
    float *L32, *C32, *M32, *W32, *D0, *D1, *z32;
    double *d_Lco;
    const std::vector<float> L32v = to32(Linv), C32v = to32(Cin), M32v = to32(Mp), W32v = to32(w);
    if ((rc = bupload(c, &L32, L32v, st)) || (rc = bupload(c, &C32, C32v, st)) || (rc = bupload(c, &M32, M32v, st)) ||
        (rc = bupload(c, &W32, W32v, st)) ||
        (rc = bupload(c, &d_Lco, Lcov, st)) || (rc = balloc(c, &D0, nPsi, st)) || (rc = balloc(c, &D1, nPsi, st)) ||
        (rc = balloc(c, &z32, nPsi, st)))
      return rc;
    BCK(cudaStreamSynchronize(st));  // host vectors of the uploads go out of scope
    d.Linv32 = L32; d.Cin32 = C32; d.Mp32 = M32; d.w32 = W32; d.Lco = d_Lco;
    d.D0 = D0; d.D1 = D1; d.z32 = z32;
    d.cvec = tc;  // the mixed form keeps c itself where the FP64 form keeps Linv c
    unsigned *fl;
    if ((rc = balloc(c, &fl, 2, st))) return rc;
    c.if_flags = fl;
  }
  // ---- autotune the sweep of this class (CUDA events over a few sweeps):
  // the shared-memory sweep over cb cells, or the register sweep with np
  // angles per thread over cb cells
  std::vector<std::pair<int, int>> cands;  // (np, cb)
  for (int cb : {32, 64, 128})
    if (cb * G <= 256 && (c.mixed ? b_mx_smem(N, G, cb) : b_sweep_smem(N, G, cb)) <= 100 * 1024)
      cands.emplace_back(0, cb);
  for (int np : {2, 4, 8}) {
    if (N % np) continue;
    const int P = N / np;
    for (int cb = kMinTile; cb <= 128; cb *= 2)
      if (cb * G * P <= 256 && cb * G * P >= 64 && (cb * G * P) % 32 == 0) cands.emplace_back(np, cb);
  }
  if (cands.empty()) cands.emplace_back(0, 32);
  std::pair<int, int> best = cands.back();
  const char *at = hook_env("OCI_AUTOTUNE");
  if (cands.size() > 1 && !(at && at[0] == '0')) {
    for (int i = 0; i < c.d.n_slabs; i++) {
      DevState &x = B.h_ds[c.slab0 + i];
      x.done = 0;
      x.cur = 0;
      x.refine = 0;
      x.blk_i = 0;  // the mixed inner sweep starts from a zero correction
      x.dcur = 0;
    }
    BCK(cudaMemcpyAsync(B.ds + c.slab0, B.h_ds + c.slab0, sizeof(DevState) * c.d.n_slabs, cudaMemcpyHostToDevice, st));
    float best_ms = 1e30f;
    for (auto cand : cands) {
      if ((rc = build_tiles(c, cand.first, cand.second, d_ts, d_tf, d_t0, d_t1, st))) return rc;
      auto sweep = [&]() {
        if (c.mixed) launch_b_mx_inner(c, B.ds + c.slab0, st);
        else launch_b_sweep(c, B.ds + c.slab0, st);
      };
      sweep();
      BCK(cudaEventRecord(B.ev0, st));
      for (int r = 0; r < 3; r++) sweep();
      BCK(cudaEventRecord(B.ev1, st));
      BCK(cudaEventSynchronize(B.ev1));
      BCK(cudaGetLastError());
      float ms = 0.f;
      cudaEventElapsedTime(&ms, B.ev0, B.ev1);
      if (ms < best_ms) {
        best_ms = ms;
        best = cand;
      }
    }
    BCK(cudaMemsetAsync(Psi0, 0, nPsi * 8, st));
    BCK(cudaMemsetAsync(Psi1, 0, nPsi * 8, st));
    if (c.mixed) {
      BCK(cudaMemsetAsync(c.d.D0, 0, nPsi * 4, st));
      BCK(cudaMemsetAsync(c.d.D1, 0, nPsi * 4, st));
    }
    for (int i = 0; i < c.d.n_slabs; i++) B.h_ds[c.slab0 + i].done = 1;
    BCK(cudaMemcpyAsync(B.ds + c.slab0, B.h_ds + c.slab0, sizeof(DevState) * c.d.n_slabs, cudaMemcpyHostToDevice, st));
  }
  // "np,cb" in OCI_BATCH_SWEEP forces a sweep shape (tests and profiling) where
  // it is valid for the class: np = 0 or np | N; cb a power of two in
  // [kMinTile, 128]; whole warps (the reductions shuffle over full warps), at
  // most 256 threads; shared memory within the set limit
  const char *force = hook_env("OCI_BATCH_SWEEP");
  if (force) {
    int fnp = -1, fcb = -1;
    if (sscanf(force, "%d,%d", &fnp, &fcb) == 2 && fcb >= kMinTile && fcb <= 128 && (fcb & (fcb - 1)) == 0) {
      bool ok;
      if (fnp == 0)
        ok = fcb * G <= 256 && (fcb * G) % 32 == 0 &&
             (c.mixed ? b_mx_smem(N, G, fcb) : b_sweep_smem(N, G, fcb)) <= 200 * 1024;
      else
        ok = (fnp == 2 || fnp == 4 || fnp == 8) && N % fnp == 0 && fcb * G * (N / fnp) <= 256 &&
             (fcb * G * (N / fnp)) % 32 == 0;
      if (ok) best = std::make_pair(fnp, fcb);
    }
  }
  return build_tiles(c, best.first, best.second, d_ts, d_tf, d_t0, d_t1, st);
}

// One body of the batched convergence loop on the classes' streams (one sweep
// of every unconverged slab, its stop rule, and for the mixed form the FP64
// refinement of the slabs that asked for it).
static void launch_batch_body(Batch &B, const std::vector<cudaStream_t> &br, cudaGraphConditionalHandle cond,
                              int use_cond) {
  for (size_t i = 0; i < B.cls.size(); i++) {
    BatchClass &c = B.cls[i];
    cudaStream_t st = br[i % br.size()];
    if (B.precision == OCI_FP64) {
      launch_b_sweep(c, B.ds + c.slab0, st);
      launch_b_finalize(c, B.ds + c.slab0, B.active, use_cond, cond, st);
    } else {
      launch_b_mx_inner(c, B.ds + c.slab0, st);
      launch_b_mx_finalize(c, B.ds + c.slab0, B.active, use_cond, cond, st);
      launch_b_mx_outer(c, B.ds + c.slab0, 1, st);
    }
  }
}

static int build_batch_graph(Batch &B) {
  cudaGraph_t graph;
  BCK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  BCK(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  BCK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  // The classes are independent until the loop test: capture each class's
  // sweep and finalize as its own branch (fork/join through events) so that
  // classes with few unconverged slabs share the GPU instead of running in turn.
  const int nc = (int)B.cls.size();
  std::vector<cudaStream_t> br(nc, nullptr);
  std::vector<cudaEvent_t> join(nc, nullptr);
  cudaEvent_t fork = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int i = 0; i < nc && e == cudaSuccess; i++) {
    e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(br[0], body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaEventRecord(fork, br[0]);
    for (int i = 1; i < nc; i++) cudaStreamWaitEvent(br[i], fork, 0);
    if (B.precision == OCI_FP64) {
      launch_batch_body(B, br, cond, 1);
    } else {
      // per class: inner sweep, finalize (sets the class's IF), IF { refinement }
      std::vector<cudaGraph_t> ifbodies(nc, nullptr);
      for (int i = 0; i < nc && e == cudaSuccess; i++) {
        BatchClass &c = B.cls[i];
        cudaStreamCaptureStatus cst;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(br[i], &cst, nullptr, &cg, nullptr, nullptr, nullptr);
        cudaGraphConditionalHandle h_if{};
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_if, cg, 0, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) break;
        c.if_handle = (unsigned long long)h_if;
        launch_b_mx_inner(c, B.ds + c.slab0, br[i]);
        launch_b_mx_finalize(c, B.ds + c.slab0, B.active, 1, cond, br[i]);
        e = cudaStreamGetCaptureInfo(br[i], &cst, nullptr, &cg, &deps, nullptr, &nd);
        cudaGraphNodeParams ip = {};
        cudaGraphNode_t ifn;
        if (e == cudaSuccess) {
          ip.type = cudaGraphNodeTypeConditional;
          ip.conditional.handle = h_if;
          ip.conditional.type = cudaGraphCondTypeIf;
          ip.conditional.size = 1;
          e = cudaGraphAddNode(&ifn, cg, deps, nullptr, nd, &ip);
        }
        if (e == cudaSuccess)
          e = cudaStreamUpdateCaptureDependencies(br[i], &ifn, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess) ifbodies[i] = ip.conditional.phGraph_out[0];
      }
      // the refinement kernels go into the IF bodies after the main capture ends
      B.if_bodies = ifbodies;
    }
    for (int i = 1; i < nc; i++) {
      cudaEventRecord(join[i], br[i]);
      cudaStreamWaitEvent(br[0], join[i], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(br[0], &body);
    if (e == cudaSuccess) e = e2;
    for (int i = 0; i < nc && e == cudaSuccess && B.precision != OCI_FP64; i++) {
      cudaGraph_t ib = B.if_bodies[i];
      e = cudaStreamBeginCaptureToGraph(br[i], ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        BatchClass &c = B.cls[i];
        launch_b_mx_outer(c, B.ds + c.slab0, 1, br[i]);
        e = cudaStreamEndCapture(br[i], &ib);
      }
    }
  }
  for (int i = 0; i < nc; i++) {
    if (br[i]) cudaStreamDestroy(br[i]);
    if (join[i]) cudaEventDestroy(join[i]);
  }
  if (fork) cudaEventDestroy(fork);
  if (e != cudaSuccess) {
    // A capture that failed inside a conditional node's body leaves the parent
    // graph in a state that the driver does not survive destroying (a failed
    // kernel launch there crashed the process in cudaGraphDestroy): the graph
    // is left to the process's exit and the error is returned.
    return cuda_fail(e, "capturing the batched convergence loop");
  }
  e = cudaGraphInstantiate(&B.graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(batch)");
  return OCI_OK;
}

void free_batch(Batch *B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  for (auto &c : B->cls)
    for (void *p : c.allocs) cudaFree(p);
  if (B->ds) cudaFree(B->ds);
  if (B->active) cudaFree(B->active);
  if (B->stage) cudaFree(B->stage);
  if (B->h_ds) cudaFreeHost(B->h_ds);
  if (B->h_bal) cudaFreeHost(B->h_bal);
  if (B->h_active) cudaFreeHost(B->h_active);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  if (B->ev0) cudaEventDestroy(B->ev0);
  if (B->ev1) cudaEventDestroy(B->ev1);
  delete B;
}

static int batch_setup(const oci_problem *probs, int n, Batch &B) {
  B.n = n;
  B.stream = (cudaStream_t)probs[0].stream;
  B.precision = probs[0].precision;
  std::map<std::pair<int, int>, int> key;
  size_t stage = 0;
  for (int s = 0; s < n; s++) {
    const oci_problem &p = probs[s];
    B.J.push_back(p.J);
    B.N.push_back(p.N);
    B.G.push_back(p.G);
    B.max_iter.push_back(p.max_iter);
    B.tol.push_back(p.tol);
    B.dt.push_back(p.dt);
    B.t.push_back(0.0);
    stage = std::max(stage, (size_t)p.J * p.G * p.N * 4);
    auto k = std::make_pair(p.N, p.G);
    auto it = key.find(k);
    int ci;
    if (it == key.end()) {
      ci = (int)B.cls.size();
      key.emplace(k, ci);
      B.cls.emplace_back();
    } else {
      ci = it->second;
    }
    B.slab_class.push_back(ci);
    B.slab_local.push_back((int)B.cls[ci].slabs.size());
    B.cls[ci].slabs.push_back(s);
    B.cls[ci].mixed = B.precision != OCI_FP64;
  }
  // class-contiguous slab order for the device states
  std::vector<int> order;
  for (auto &c : B.cls) {
    c.slab0 = (int)order.size();
    for (int s : c.slabs) order.push_back(s);
  }
  BCK(cudaMalloc(&B.stage, stage * 8 + 16));
  BCK(cudaMalloc(&B.ds, sizeof(DevState) * n));
  BCK(cudaMallocHost(&B.h_ds, sizeof(DevState) * n));
  BCK(cudaMalloc(&B.active, sizeof(int)));
  BCK(cudaEventCreate(&B.ev0));
  BCK(cudaEventCreate(&B.ev1));
  std::memset(B.h_ds, 0, sizeof(DevState) * n);
  for (int i = 0; i < n; i++) B.h_ds[i].done = 1;
  BCK(cudaMemcpyAsync(B.ds, B.h_ds, sizeof(DevState) * n, cudaMemcpyHostToDevice, B.stream));
  BCK(cudaFuncSetAttribute(k_b_sweep_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  BCK(cudaFuncSetAttribute(k_b_mx_inner_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  size_t nbal = 0;
  for (auto &c : B.cls) {
    int rc = setup_class(B, c, probs);
    if (rc) return rc;
    nbal += (size_t)c.d.n_slabs * c.d.G * 10;
  }
  BCK(cudaMallocHost(&B.h_bal, nbal * 8 + 16));
  BCK(cudaMallocHost(&B.h_active, sizeof(int)));
  // OCI_NO_GRAPH=1: drive the loop from the host (profilers that do not
  // descend into conditional graph bodies see every kernel)
  const char *ng = hook_env("OCI_NO_GRAPH");
  B.no_graph = ng && ng[0] == '1';
  if (!B.no_graph) {
    int rc = build_batch_graph(B);
    if (rc) return rc;
  }
  BCK(cudaStreamSynchronize(B.stream));
  BCK(cudaGetLastError());
  return OCI_OK;
}

// device-state slot of batch slab s
static inline int slot(const Batch &B, int s) { return B.cls[B.slab_class[s]].slab0 + B.slab_local[s]; }

static int batch_step(Batch &B, oci_stats *st) {
  int kmax = kBatchMxKmax;
  double theta = kBatchMxTheta;
  {
    const char *km = hook_env("OCI_MX_KMAX"), *th = hook_env("OCI_MX_THETA");
    if (km) kmax = std::max(1, atoi(km));
    if (th) theta = atof(th);
  }
  cudaStream_t s = B.stream;
  for (int i = 0; i < B.n; i++) {
    DevState &d = B.h_ds[slot(B, i)];
    d.l = 0;
    d.status = OCI_OK;
    d.done = 0;
    d.fixed = 0;
    d.max_iter = B.max_iter[i];
    d.tol = B.tol[i];
    d.e = d.e_prev = d.rho = 0.0;
    d.dcur = 0;
    d.blk_i = 0;
    d.refine = 0;
    d.applied = 0;
    d.k_max = kmax;
    d.n_refine = 0;
    d.theta = theta;
    d.e_blk0 = 0.0;
    d.inplace = 0;
  }
  BCK(cudaMemcpyAsync(B.ds, B.h_ds, sizeof(DevState) * B.n, cudaMemcpyHostToDevice, s));
  const int active = B.n;
  BCK(cudaMemcpyAsync(B.active, &active, sizeof(int), cudaMemcpyHostToDevice, s));
  const bool mixed = B.precision != OCI_FP64;
  for (auto &c : B.cls) {
    if (mixed) {
      launch_b_mx_step_const(c, s);        // c (not pre-multiplied)
      launch_b_mx_outer(c, B.ds + c.slab0, 0, s);  // FP64 residual of the initial iterate
    } else {
      launch_b_step_const(c, s);
    }
  }
  BCK(cudaEventRecord(B.ev0, s));
  if (B.no_graph) {
    // batches of 16 bodies on the one stream, then read the unconverged count
    int cap = 0;
    for (int i = 0; i < B.n; i++) cap = std::max(cap, B.max_iter[i]);
    const std::vector<cudaStream_t> one{s};
    cudaGraphConditionalHandle none{};
    for (int done = 0; done < cap;) {
      const int nb = std::min(16, cap - done);
      for (int k = 0; k < nb; k++) launch_batch_body(B, one, none, 0);
      done += nb;
      BCK(cudaMemcpyAsync(B.h_active, B.active, sizeof(int), cudaMemcpyDeviceToHost, s));
      BCK(cudaStreamSynchronize(s));
      if (*B.h_active <= 0) break;
    }
  } else {
    BCK(cudaGraphLaunch(B.graph, s));
  }
  BCK(cudaEventRecord(B.ev1, s));
  if (mixed)
    for (auto &c : B.cls) launch_b_mx_settle(c, B.ds + c.slab0, s);
  for (auto &c : B.cls) launch_b_carry(c, B.ds + c.slab0, s);
  BCK(cudaMemcpyAsync(B.h_ds, B.ds, sizeof(DevState) * B.n, cudaMemcpyDeviceToHost, s));
  size_t off = 0;
  for (auto &c : B.cls) {
    const size_t nb = (size_t)c.d.n_slabs * c.d.G * 10;
    BCK(cudaMemcpyAsync(B.h_bal + off, c.d.bal, nb * 8, cudaMemcpyDeviceToHost, s));
    off += nb;
  }
  BCK(cudaStreamSynchronize(s));
  BCK(cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, B.ev0, B.ev1);
  int worst = OCI_OK;
  off = 0;
  std::vector<size_t> cls_off;
  for (auto &c : B.cls) {
    cls_off.push_back(off);
    off += (size_t)c.d.n_slabs * c.d.G * 10;
  }
  for (int i = 0; i < B.n; i++) {
    const DevState &d = B.h_ds[slot(B, i)];
    if (d.status == OCI_OK) B.t[i] += B.dt[i];
    else if (worst == OCI_OK) worst = d.status;
    if (!st) continue;
    oci_stats &o = st[i];
    o.iters = d.l;
    o.status = d.status;
    o.e_last = d.e;
    o.rho_e_last = d.rho;
    o.t = B.t[i];
    o.seconds = ms * 1e-3;
    o.refinements = B.precision == OCI_FP64 ? 0 : d.n_refine;
    o.reserved = 0;
    o.balance_rel[0] = o.balance_rel[1] = 0.0;
    if (d.status != OCI_OK) continue;
    const int ci = B.slab_class[i], G = B.G[i];
    const double *bal = B.h_bal + cls_off[ci] + (size_t)B.slab_local[i] * G * 10;
    for (int g = 0; g < G; g++)
      for (int b = 0; b < 2; b++) {
        const double *x = bal + g * 10 + b * 5;
        const double r = x[0] + x[1] + x[2] - x[3] - x[4];
        const double sc = fabs(x[0]) + fabs(x[1]) + fabs(x[2]) + fabs(x[3]) + fabs(x[4]);
        const double rel = sc > 0 ? fabs(r) / sc : 0.0;
        if (rel > o.balance_rel[b]) o.balance_rel[b] = rel;
      }
  }
  if (worst != OCI_OK) set_error("at least one slab of the batch did not converge (see its stats)");
  return worst;
}

static int batch_get(const Batch &B, int s, int what, double *out) {
  if (s < 0 || s >= B.n) return set_error("slab index out of range"), OCI_E_INVAL;
  if (!out) return set_error("output is NULL"), OCI_E_INVAL;
  const BatchClass &c = B.cls[B.slab_class[s]];
  const int i = B.slab_local[s];
  const int J = c.h_J[i], N = c.d.N, G = c.d.G;
  const DevState &d = B.h_ds[slot(B, s)];
  const double *src;
  int K;
  if (what == 0) {
    src = (d.cur ? c.d.Psi1 : c.d.Psi0) + c.h_start[i];
    K = G * N * 4;
  } else if (what == 1) {
    src = c.d.phi + c.h_start[i];
    K = G * 4;
  } else {
    BCK(cudaMemcpyAsync(out, c.d.bal + (size_t)i * G * 10, (size_t)G * 10 * 8, cudaMemcpyDefault, B.stream));
    BCK(cudaStreamSynchronize(B.stream));
    return OCI_OK;
  }
  k_bt_out<<<dim3((J + 255) / 256, K), 256, 0, B.stream>>>(J, c.d.Jc, K, src, B.stage);
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(out, B.stage, (size_t)J * K * 8, cudaMemcpyDefault, B.stream));
  BCK(cudaStreamSynchronize(B.stream));
  return OCI_OK;
}

}  // namespace oci

using namespace oci;

extern "C" {

int oci_batch_setup(const oci_problem *probs, int32_t n, oci_handle **out) {
  if (!out) return set_error("out is NULL"), OCI_E_INVAL;
  *out = nullptr;
  if (!probs || n < 1) return set_error("need at least one problem"), OCI_E_INVAL;
  for (int s = 0; s < n; s++) {
    int rc = validate(&probs[s]);
    if (rc) return rc;
    if ((probs[s].precision != OCI_FP64 && probs[s].precision != OCI_FP32_IR) ||
        probs[s].solver == OCI_SOLVER_DENSE_LU || probs[s].guess != OCI_GUESS_PREV)
      return set_error("the batched form is FP64 or FP32_IR, structured solver, GUESS_PREV"), OCI_E_INVAL;
    if (probs[s].precision != probs[0].precision)
      return set_error("all slabs of a batch share one precision"), OCI_E_INVAL;
    if (probs[s].stream != probs[0].stream) return set_error("all slabs of a batch share one stream"), OCI_E_INVAL;
  }
  oci_handle *h = new (std::nothrow) oci_handle();
  if (!h) return set_error("host allocation failed"), OCI_E_NOMEM;
  h->batch = new (std::nothrow) Batch();
  int rc = h->batch ? batch_setup(probs, n, *h->batch) : OCI_E_NOMEM;
  if (rc) {
    oci_destroy(h);
    return rc;
  }
  *out = h;
  set_error("");
  return OCI_OK;
}

int oci_batch_step(oci_handle *h, oci_stats *st) {
  if (!h || !h->batch) return set_error("not a batched handle"), OCI_E_INVAL;
  return batch_step(*h->batch, st);
}

int oci_batch_size(const oci_handle *h, int32_t *n) {
  if (!h || !h->batch || !n) return set_error("not a batched handle"), OCI_E_INVAL;
  *n = h->batch->n;
  return OCI_OK;
}

int oci_batch_get_psi(const oci_handle *h, int32_t s, double *psi) {
  if (!h || !h->batch) return set_error("not a batched handle"), OCI_E_INVAL;
  return batch_get(*h->batch, s, 0, psi);
}

int oci_batch_get_phi(const oci_handle *h, int32_t s, double *phi) {
  if (!h || !h->batch) return set_error("not a batched handle"), OCI_E_INVAL;
  return batch_get(*h->batch, s, 1, phi);
}

int oci_batch_get_balance(const oci_handle *h, int32_t s, double *bal) {
  if (!h || !h->batch) return set_error("not a batched handle"), OCI_E_INVAL;
  return batch_get(*h->batch, s, 2, bal);
}

}  // extern "C"
