// oci_batch.h -- batched form: device view of one (N, G) class of slabs and the
// host-side batch handle (not part of the ABI).
#pragma once
#include <vector>

#include "oci_internal.h"

namespace oci {

// Plain-pointer view of one class, passed by value to the kernels.
struct BatchClassDev {
  int N, G, Jc, n_tiles, n_slabs;
  const int32_t *type;             // [Jc] class-wide cell-type id
  const int32_t *seg;              // [Jc] class-local slab index, -1 for padding
  const int32_t *slab_start;       // [n_slabs] first cell
  const int32_t *slab_J;           // [n_slabs] cells
  const int32_t *slab_tile0;       // [n_slabs] first tile
  const int32_t *slab_tile1;       // [n_slabs] one past the last tile
  const int32_t *tile_slab;        // [n_tiles]
  const int32_t *tile_first_cell;  // [n_tiles]
  const double *Linv, *Cin, *Mp, *Kap, *tdx, *tsig;  // per type, as TypeTables
  const double *tah;               // [T][G] dx / (2 v_g dt) of the type's slab
  const double *w, *mu;            // [N]
  const double *inc;               // [n_slabs][2][G][N][2]
  const double *Q;                 // [G][4][Jc] or NULL
  double *Psi0, *Psi1, *tc, *psi_prev, *phi;
  double *partials;                // [n_tiles]
  double *bal_partials;            // [Jc/32][G][8]
  double *bal;                     // [n_slabs][G][10]
  // mixed-precision form (FP32 inner sweeps on a correction, FP64 refinement)
  float *D0, *D1, *z32;            // [G][N][4][Jc]
  double *cvec;                    // [G][N][4][Jc] per-step constant c (not pre-multiplied); aliases tc
  const float *Linv32, *Cin32, *Mp32, *w32;
  const double *Lco;               // [T][G][N][5] {a, mu/2, alpha/2, alpha, alpha+a}
};

struct BatchClass {
  BatchClassDev d{};
  bool mixed = false;
  unsigned *if_flags = nullptr;         // mixed form in the graph: {any slab refines, blocks done}
  unsigned long long if_handle = 0;     // IF node of the class's refinement kernel
  int cb = 128;     // cells per tile (autotuned)
  int np = 0;       // angles per thread of the register sweep; 0 = shared-memory sweep (autotuned)
  int grid = 0;     // persistent grid size
  int slab0 = 0;    // index of the class's first slab in the batch
  std::vector<int> slabs;  // batch slab index of each class-local slab
  std::vector<int> h_start, h_J;
  std::vector<void *> allocs;
};

struct Batch {
  int n = 0;
  int precision = OCI_FP64;
  std::vector<BatchClass> cls;
  std::vector<int> slab_class, slab_local;  // batch slab -> (class, local index)
  std::vector<int> J, N, G, max_iter;
  std::vector<double> tol, dt, t;
  DevState *ds = nullptr;     // [n] device
  DevState *h_ds = nullptr;   // [n] pinned
  int *active = nullptr;      // device counter of unconverged slabs
  double *h_bal = nullptr;    // pinned, per class concatenated
  int *h_active = nullptr;    // pinned copy of the unconverged count (host-driven loop)
  bool no_graph = false;      // drive the loop from the host (OCI_NO_GRAPH=1)
  std::vector<cudaGraph_t> if_bodies;  // mixed form: per-class IF bodies while the graph is built
  cudaStream_t stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double *stage = nullptr;    // device staging, largest slab Psi
};

size_t b_sweep_smem(int N, int G, int cb);
int b_max_grid(int N, int G, int cb);
void launch_b_step_const(BatchClass &c, cudaStream_t st);
void launch_b_sweep(BatchClass &c, DevState *ds, cudaStream_t st);
void launch_b_finalize(BatchClass &c, DevState *ds, int *active, int use_cond, cudaGraphConditionalHandle cond,
                       cudaStream_t st);
void launch_b_carry(BatchClass &c, DevState *ds, cudaStream_t st);
const void *k_b_sweep_ptr();
// mixed-precision batched form
void launch_b_mx_step_const(BatchClass &c, cudaStream_t st);
void launch_b_mx_inner(BatchClass &c, DevState *ds, cudaStream_t st);
void launch_b_mx_finalize(BatchClass &c, DevState *ds, int *active, int use_cond, cudaGraphConditionalHandle cond,
                          cudaStream_t st);
void launch_b_mx_outer(BatchClass &c, DevState *ds, int mode, cudaStream_t st);
void launch_b_mx_settle(BatchClass &c, DevState *ds, cudaStream_t st);
size_t b_mx_smem(int N, int G, int cb);
int b_mx_max_grid(int N, int G, int cb);
// register sweep (angles split over N/np threads per cell; FP64 or the FP32 inner sweep)
size_t b_reg_smem(int N, int G, int cb, int np, int es);
int b_reg_max_grid(int N, int G, int cb, int np, bool mixed);
const void *k_b_reg_ptr(int np, bool mixed);
const void *k_b_mx_inner_ptr();

}  // namespace oci
