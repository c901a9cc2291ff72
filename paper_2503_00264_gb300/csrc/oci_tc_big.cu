// oci_tc_big.cu -- tcgen05 block apply of the TF32 / BF16x3 mixed forms, for any
// number of unknowns per cell up to 4NG = 512 (e.g. S16 with 8 groups).
//
// The inner sweep of the mixed forms is delta^{i+1} = A~^{-1} (r + B delta^i) per
// cell (where cells share material, width and dt, the inverse of the cell
// matrix of Eqs. Aj, scatter, fullOCIlhs is applied to all of their right-hand
// sides as one dense GEMM).  For a tile of 128 cells of one type this is,
// transposed so that the cells are the MMA's M and the unknowns its N,
//   D[128 cells x n] = RHS[128 cells x n] . (A^{-1})^T,      n = 4NG <= 512,
// with the accumulator in tensor memory (lane = cell, column = unknown; n
// columns).  The inverse (1 MB per type in TF32 at n = 512) does not fit in
// shared memory, so the K dimension is walked in chunks of 16:
//   - per chunk one 1D bulk copy per N-tile of 256 unknowns brings that chunk of
//     A^{-1} (stored chunk by chunk in the K-major no-swizzle canonical layout)
//     into a stage of shared memory, and two 2D tensor copies bring rows
//     k .. k+15 of r and of the old correction (with a halo of 4 cells each side
//     for the neighbours' inflow) into one of three input buffers;
//   - eight builder warps form that chunk of the RHS (r + B delta, FP32 -> TF32
//     or BF16 hi/lo) in the stage next to the A^{-1} chunk;
//   - one thread of a control warp issues the chunk's MMAs (M = 128 cells,
//     N <= 256 unknowns per N-tile) and commits them to the stage's mbarrier;
//     one thread of a second control warp issues the copies: a chunk's inputs
//     as soon as the builders have consumed the buffer three chunks back, its
//     A^{-1} chunk as soon as the MMAs three chunks back have freed the stage
//     (three stages);
//   - after the last chunk of a tile the builder warps drain the accumulators
//     (tcgen05.ld: one register per unknown, one lane per cell), form delta
//     and the FP32 norm partial; loads and stores are 128-byte rows of 32 cells.
// Coupling form (n a multiple of 32): r is the same for every inner sweep
// of a refinement block, so the block's first sweep (zero old correction, the
// full form above) also stores z = A~^{-1} r, and every later sweep computes
//   delta = z + U . (A~^{-1} B)^T
// over the n/2 inflow columns only (B delta puts |mu| times an upstream corner of
// the neighbour into two rows of each (group, angle) block): half the K-chunks,
// a builder step that only gathers the upstream corners, and z added in the drain.
// One CTA per SM walks the tiles persistently; a tile whose cells are of more
// than one type (a region boundary inside it) is taken once per type, each pass
// keeping only its own cells (work items (tile, type), a separate instantiation).
// The norm, the stop rule and the refinement decision are fused into the last
// CTA to finish.  Every wait is
// bounded: on a timeout the CTA waits (bounded) for its copies and MMAs in
// flight, frees its tensor memory and records OCI_E_TIMEOUT.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "oci_device.cuh"
#include "oci_internal.h"

namespace oci {

constexpr int kBigM = 128;         // MMA M: cells per tile
constexpr int kBigN = 128;         // cells per tile (the M of the MMA)
constexpr int kBigNT = 256;        // MMA N: unknowns per N-tile
constexpr int kBigKC = 16;         // K elements per chunk
constexpr int kBigABlk = 16384;    // one chunk of A^{-1} for one N-tile: 256 rows x 16 K (TF32, or BF16 hi + lo)
constexpr int kBigRBlk = 8192;     // one chunk of the RHS: 128 cells x 16 K (TF32, or BF16 hi + lo)
constexpr int kBigStages = 3;      // A^{-1} + RHS stages
constexpr int kBigBuilders = 256;  // eight warps: RHS builders and drain
constexpr int kBigThreads = kBigBuilders + 64;  // and two control warps: MMAs, copies
constexpr long long kBigSpin = 1 << 22;
constexpr int kBigHalo = 4;                                 // columns each side of the delta box (16 B)
constexpr int kBigDW = kBigN + 2 * kBigHalo;                // delta box width
constexpr int kBigInFull = kBigKC * (kBigN + kBigDW) * 4;   // full form: r box + delta box of one chunk
constexpr int kBigInHalf = 2 * kBigKC * kBigDW * 4;         // coupling form: delta box of 32 rows
constexpr int kBigInBytes = kBigInFull > kBigInHalf ? kBigInFull : kBigInHalf;
// Input buffers: a chunk's copies are issued once the builders have consumed the
// buffer kBigInBuf chunks back, so the builders can be at most kBigInBuf chunks
// ahead of the copy thread's wait on rhs_full; with more buffers than stages they
// could complete the same stage's next phase before that wait and it would miss
// a phase.  Hence kBigInBuf <= kBigStages.
constexpr int kBigInBuf = 3;
constexpr int kBigStash = 256;  // first tensor-memory column of the old correction (n <= 256)
static_assert(kBigInBuf <= kBigStages, "input buffers must not outnumber the stages");

namespace {

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bounded wait for the phase of parity `parity` of an mbarrier.
__device__ __forceinline__ bool big_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok = 0;
  for (long long it = 0; it < kBigSpin && !ok; it++) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (!ok) __nanosleep(32);
  }
  return ok != 0;
}

// Shared-memory matrix descriptor: K-major, no swizzle (version 1 for tcgen05).
__device__ __forceinline__ uint64_t big_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

}  // namespace

// Byte offset of (row, k) inside one chunk block of [rows x 32 K]: 8-row x
// 16-byte core matrices, adjacent along K 128 B apart (LBO), 8-row groups
// (32 * es / 16) * 128 B apart (SBO).
__host__ __device__ inline uint32_t big_off(int row, int k, int es) {
  const int kc4 = 16 / es;
  return (uint32_t)((row >> 3) * (kBigKC * es / 16) * 128 + (k / kc4) * 128 + (row & 7) * 16 + (k % kc4) * es);
}

// KIND: 1 = TF32, 2 = BF16 x3.  MIXED: some tile holds cells of more than one type
// (work items from `items`); otherwise item i of a CTA is its i-th tile and
// `items` is not read.
template <int KIND, bool MIXED>
__global__ void __launch_bounds__(kBigThreads, 1) k_tc_big(
    const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmD0,
    const __grid_constant__ CUtensorMap tmD1, int J, int Jp, int N, int G, int NT, int NK,
    const int32_t *__restrict__ type, const unsigned char *__restrict__ Aimg, const float *__restrict__ mu,
    const float *__restrict__ r32, float *D0, float *D1, DevState *ds, double *__restrict__ partials,
    unsigned *counter, double *e_hist, cudaGraphConditionalHandle cond, int use_cond,
    const int2 *__restrict__ items, int n_items, const unsigned char *__restrict__ AimgH, int NKH, float *Zt) {
  extern __shared__ __align__(1024) unsigned char smb_[];
  // a_full: a stage's A^{-1} chunk has landed; rhs_full: the eight builder warps
  // have written a stage's RHS chunk; mma_done: a stage's MMAs have completed;
  // in_full: an input buffer's r / delta boxes have landed; tmem_empty: the
  // accumulators of the last tile have been drained
  __shared__ __align__(8) uint64_t a_full[kBigStages], rhs_full[kBigStages], mma_done[kBigStages], in_full[kBigInBuf],
      tmem_empty;
  __shared__ uint32_t tslot;
  __shared__ float mu_s[kMaxN];
  __shared__ double red[kBigThreads / 32];
  __shared__ bool s_last;
  __shared__ int s_fail;
  constexpr int es = KIND == 1 ? 4 : 2;
  constexpr int apart = kBigABlk / 2;  // BF16: the lo image follows the hi image
  constexpr int rpart = kBigRBlk / 2;
  constexpr int ksteps = kBigKC * es / 32;  // MMAs per chunk, N-tile and pass (K = 8 TF32 / 16 BF16)
  constexpr int npass = KIND == 1 ? 1 : 3;  // BF16 x3: hi.hi + lo.hi + hi.lo
  const int n = 4 * N * G;
  unsigned char *sm = (unsigned char *)(((uintptr_t)smb_ + 1023) & ~(uintptr_t)1023);
  const size_t stage_bytes = (size_t)NT * kBigABlk + kBigRBlk;  // NT A^{-1} blocks, then the RHS block
  unsigned char *in_base = sm + kBigStages * stage_bytes;        // kBigInBuf input buffers
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (ds->done) return;  // uniform
  const bool zero = ds->refine || ds->blk_i == 0;
  // coupling form (an image of the inflow columns is present, and this is not the
  // first sweep of a refinement block): D = U . (A~^{-1} B)^T over the n/2 inflow
  // columns, delta = z + D with z = A~^{-1} r kept from the block's first sweep
  const bool half = !zero && AimgH != nullptr;
  const int NKe = half ? NKH : NK;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  // one column per unknown; with n <= 256 the old correction of the tile's cells is
  // also kept in tensor memory (columns kBigStash ..), stored by the builders as the
  // chunks arrive, so the drain reads it there instead of from HBM
  const uint32_t cols = 512u;
  const bool stash = n <= kBigNT;
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    for (int q = 0; q < kBigStages; q++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&a_full[q])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&rhs_full[q])), "r"(kBigBuilders / 32));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mma_done[q])), "r"(1));
    }
    for (int q = 0; q < kBigInBuf; q++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&in_full[q])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&tmem_empty)), "r"(kBigBuilders / 32));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  for (int i = t; i < N; i += kBigThreads) mu_s[i] = mu[i];
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  // work items (tile, cell type): one per tile, or one per type present in a tile
  // whose cells are not all of one type (then bit 30 of the type word is set); the
  // CTA's i-th item is items[blockIdx.x + i gridDim.x]
  const int my_items = (int)blockIdx.x < n_items ? (n_items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int n_chunks = my_items * NKe;  // chunk g: the CTA's item g / NKe, K-chunk g % NKe
  const int N2 = N / 2;
  float e2 = 0.f;
  bool failed = false;

  if (w < kBigBuilders / 32) {
    // ------------------------------------------------ builders (and drain)
    const int c = t & (kBigN - 1), hh = t >> 7;  // cell c, rows hh*8 .. hh*8+7 of a chunk
    int it = blockIdx.x;
    int2 wi = make_int2((int)blockIdx.x, 0), wn = wi;
    if (MIXED && my_items > 0) wi = wn = items[it];
    bool keep = true;  // the drained cell of this thread is of the item's type
    for (int g = 0, kc = 0, tile = wi.x, s = 0, u3 = 0; g < n_chunks; g++) {
      if (MIXED && kc == 0) {  // loads for this item's drain and the next item, well ahead of their use
        if (it + (int)gridDim.x < n_items) wn = items[it + gridDim.x];
        const int jd = tile * kBigN + 32 * (w & 3) + lane;
        keep = !(wi.y >> 30) || (jd < J && type[jd] == (wi.y & 0x3FFFFFFF));
      }
      const int ib = g % kBigInBuf;
      float *in_r = (float *)(in_base + (size_t)ib * kBigInBytes);  // full form: r [16][128]
      float *in_d = half ? in_r : in_r + kBigKC * kBigN;             // delta [16][136], coupling form [32][136]
      unsigned char *stB = sm + (size_t)s * stage_bytes + (size_t)NT * kBigABlk;
      // this chunk's inputs have landed and the stage's MMAs of chunk g - 3 are done; a new
      // tile's old-correction copy in tensor memory waits until every builder warp has
      // drained the previous tile (a warp drains columns its partner warp stored)
      bool ok = big_wait(su32(&in_full[ib]), (uint32_t)((g / kBigInBuf) & 1));
      if (ok && g >= kBigStages) ok = big_wait(su32(&mma_done[s]), (uint32_t)((u3 - 1) & 1));
      if (ok && stash && kc == 0 && g > 0) {
        ok = big_wait(su32(&tmem_empty), (uint32_t)(((g / NKe) - 1) & 1));
        asm volatile("tcgen05.fence::after_thread_sync;");
      }
      if (!__all_sync(0xffffffffu, ok)) {  // warp-uniform: the warp leaves together
        s_fail = 1;
        failed = true;
        break;
      }
      {  // RHS of cell c, K rows hh*8 .. hh*8+7 of this chunk: TF32, or BF16 hi / lo
        const int j = tile * kBigN + c;
        const bool act = j < J;
        float v[8];
        if (half) {
          // coupling form: K column 2 (gN + m) + s is the inflow of (group, angle) gN + m
          // (s = 0 time average, 1 time edge): for mu > 0 corner 2s + 1 (R) of cell j-1,
          // for mu < 0 corner 2s (L) of cell j+1 (|mu| is in the image).  The chunk's box
          // holds the 32 unknowns of the (g, m) blocks 8 kc .. 8 kc + 7.
          const bool has_l = act && j > 0, has_r = act && j < J - 1;
          int m = (kc * 8 + hh * 4) % N;
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int ql = hh * 4 + q;
            const bool pos = m >= N2;
#pragma unroll
            for (int sc = 0; sc < 2; sc++) {
              const float up = in_d[(4 * ql + 2 * sc + 1) * kBigDW + c + kBigHalo - 1];
              const float dn = in_d[(4 * ql + 2 * sc) * kBigDW + c + kBigHalo + 1];
              v[2 * q + sc] = pos ? (has_l ? up : 0.f) : (has_r ? dn : 0.f);
            }
            m = m + 1 == N ? 0 : m + 1;
          }
        } else {
          // full form, r + B delta: all shared-memory loads first (no branch between
          // them), then the inflow terms: rows kc*16 + hh*8 .. +7 are two (group, angle)
          // blocks of four corners; for mu > 0 the even rows take mu * (R corner of cell
          // j-1), for mu < 0 the odd rows |mu| * (L corner of cell j+1)
          float up[4], dn[4];
#pragma unroll
          for (int i = 0; i < 8; i++) v[i] = in_r[(hh * 8 + i) * kBigN + c];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int kl2 = hh * 8 + 2 * q;
            up[q] = in_d[(kl2 + 1) * kBigDW + c + kBigHalo - 1];
            dn[q] = in_d[kl2 * kBigDW + c + kBigHalo + 1];
          }
          const int m0 = (kc * (kBigKC / 4) + hh * 2) % N;
          const int m1 = m0 + 1 == N ? 0 : m0 + 1;
          const float mf0 = mu_s[m0], mf1 = mu_s[m1];
          const bool lag = act && !zero;
          const bool has_l = lag && j > 0, has_r = lag && j < J - 1;
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int m = q < 2 ? m0 : m1;
            const float mf = q < 2 ? mf0 : mf1;
            const bool pos = m >= N2;
            v[2 * q] = fmaf(mf, (pos && has_l) ? up[q] : 0.f, v[2 * q]);
            v[2 * q + 1] = fmaf(-mf, (!pos && has_r) ? dn[q] : 0.f, v[2 * q + 1]);
          }
          if (!act) {
#pragma unroll
            for (int i = 0; i < 8; i++) v[i] = 0.f;
          }
        }
        if (KIND == 1) {
          *(float4 *)(stB + big_off(c, hh * 8, 4)) = make_float4(v[0], v[1], v[2], v[3]);
          *(float4 *)(stB + big_off(c, hh * 8 + 4, 4)) = make_float4(v[4], v[5], v[6], v[7]);
        } else {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const float a0 = v[2 * i], a1 = v[2 * i + 1];
            const __nv_bfloat16 h0 = __float2bfloat16_rn(a0), h1 = __float2bfloat16_rn(a1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(a0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(a1 - __bfloat162float(h1));
            hi[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lo[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
          }
          const uint32_t off = big_off(c, hh * 8, 2);
          *(uint4 *)(stB + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *(uint4 *)(stB + rpart + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
      if (stash && half) {  // old correction of cell c, box rows hh*16 .. +15 (unknowns 32 kc + ..) -> tensor memory
        uint32_t ov[16];
#pragma unroll
        for (int i = 0; i < 16; i++) ov[i] = __float_as_uint(in_d[(hh * 16 + i) * kBigDW + c + kBigHalo]);
        const uint32_t sa = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(kBigStash + kc * 32 + hh * 16);
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(sa),
            "r"(ov[0]), "r"(ov[1]), "r"(ov[2]), "r"(ov[3]), "r"(ov[4]), "r"(ov[5]), "r"(ov[6]), "r"(ov[7]), "r"(ov[8]),
            "r"(ov[9]), "r"(ov[10]), "r"(ov[11]), "r"(ov[12]), "r"(ov[13]), "r"(ov[14]), "r"(ov[15])
            : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
      } else if (stash) {  // old correction of cell c, rows hh*8 .. hh*8+7 of this chunk -> tensor memory
        uint32_t ov[8];
#pragma unroll
        for (int i = 0; i < 8; i++) ov[i] = __float_as_uint(in_d[(hh * 8 + i) * kBigDW + c + kBigHalo]);
        const uint32_t sa = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(kBigStash + kc * kBigKC + hh * 8);
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(sa), "r"(ov[0]),
                     "r"(ov[1]), "r"(ov[2]), "r"(ov[3]), "r"(ov[4]), "r"(ov[5]), "r"(ov[6]), "r"(ov[7])
                     : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
      }
      // the RHS is visible to the tensor cores and the inputs are consumed
      asm volatile("fence.proxy.async.shared::cta;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&rhs_full[s])) : "memory");
      if (kc == NKe - 1) {
        // last chunk of the tile: drain the accumulators once its MMAs are done.  Warp
        // w reads the lanes (cells) 32 (w % 4) .. +31; the n columns (unknowns) go in
        // blocks of 32 to the two warps of a lane quarter alternately; each register
        // of a block is one unknown of the lane's cell, so every load and store is a
        // 128-byte row of 32 cells.  The old correction of the next block is loaded
        // before this one's accumulators are read; in the coupling form z of the
        // warp's first block is loaded while the last chunk's MMAs run.
        const int q4 = w & 3, g2 = w >> 2;
        const int j = tile * kBigN + 32 * q4 + lane;
        const bool act = j < J && keep;  // only this item's cells
        const int nb = n / 32;  // column blocks
        // coupling form: z (and, above 256 unknowns, the old correction) of the warp's first
        // block into L1 while the last chunk's MMAs run
        auto prefetch_block = [&](int b_) {
          const size_t ix = (size_t)(b_ * 32) * Jp + j;
          const float *pz = Zt + ix, *pd = Din + ix;
#pragma unroll 4
          for (int i = 0; i < 32; i++, pz += Jp, pd += Jp) {
            asm volatile("prefetch.global.L1 [%0];" ::"l"(pz));
            if (!stash) asm volatile("prefetch.global.L1 [%0];" ::"l"(pd));
          }
        };
        if (half && act && g2 < nb) prefetch_block(g2);
        if (!__all_sync(0xffffffffu, big_wait(su32(&mma_done[s]), (uint32_t)(u3 & 1)))) {
          s_fail = 1;
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (half) {  // delta = z + D
          // (in half blocks of 16 columns: two tensor-memory reads and z per half; z of the
          // warp's next block is prefetched into L1 when a block starts)
#pragma unroll 1
          for (int hb = 2 * g2; hb < 2 * nb; hb += (hb & 1) ? 3 : 1) {  // halves 2 b_, 2 b_ + 1 of the warp's blocks
            if (!(hb & 1) && act && hb / 2 + 2 < nb) prefetch_block(hb / 2 + 2);
            float zc[16];
#pragma unroll
            for (int i = 0; i < 16; i++) zc[i] = act ? Zt[(size_t)(hb * 16 + i) * Jp + j] : 0.f;
            uint32_t r[16], o[16];
            const uint32_t addr = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(hb * 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(addr));
            if (stash) {  // the old correction from the builders' copy in tensor memory
              asm volatile(
                  "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                  : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]), "=r"(o[7]),
                    "=r"(o[8]), "=r"(o[9]), "=r"(o[10]), "=r"(o[11]), "=r"(o[12]), "=r"(o[13]), "=r"(o[14]),
                    "=r"(o[15])
                  : "r"(addr + (uint32_t)kBigStash));
            } else {  // from HBM (prefetched into L1 a block ahead)
#pragma unroll
              for (int i = 0; i < 16; i++) o[i] = act ? __float_as_uint(Din[(size_t)(hb * 16 + i) * Jp + j]) : 0u;
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (act) {
#pragma unroll
              for (int i = 0; i < 16; i++) {
                const float x = __uint_as_float(r[i]) + zc[i];
                const float d = x - __uint_as_float(o[i]);
                e2 = fmaf(d, d, e2);
                Dout[(size_t)(hb * 16 + i) * Jp + j] = x;
              }
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tmem_empty)) : "memory");
        } else {
          float dold[32], dnxt[32];
          const bool zt_w = zero && Zt && act;
          auto load_old = [&](int b_, float *dst) {
            if (stash) {  // from the builders' copy in tensor memory
              uint32_t o[32];
              const uint32_t oa = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(kBigStash + b_ * 32);
              asm volatile(
                  "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                  : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]), "=r"(o[7]),
                    "=r"(o[8]), "=r"(o[9]), "=r"(o[10]), "=r"(o[11]), "=r"(o[12]), "=r"(o[13]), "=r"(o[14]),
                    "=r"(o[15]), "=r"(o[16]), "=r"(o[17]), "=r"(o[18]), "=r"(o[19]), "=r"(o[20]), "=r"(o[21]),
                    "=r"(o[22]), "=r"(o[23]), "=r"(o[24]), "=r"(o[25]), "=r"(o[26]), "=r"(o[27]), "=r"(o[28]),
                    "=r"(o[29]), "=r"(o[30]), "=r"(o[31])
                  : "r"(oa));
              asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
              for (int i = 0; i < 32; i++) dst[i] = (act && !zero) ? __uint_as_float(o[i]) : 0.f;
            } else {
#pragma unroll
              for (int i = 0; i < 32; i++) dst[i] = (act && !zero) ? Din[(size_t)(b_ * 32 + i) * Jp + j] : 0.f;
            }
          };
          if (g2 < nb) load_old(g2, dold);
#pragma unroll 1
          for (int b_ = g2; b_ < nb; b_ += 2) {
            uint32_t r[32];
            const uint32_t addr = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(b_ * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(addr));
            if (b_ + 2 < nb) load_old(b_ + 2, dnxt);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (act) {
#pragma unroll
              for (int i = 0; i < 32; i++) {
                const float o = __uint_as_float(r[i]);
                const float d = o - dold[i];
                e2 = fmaf(d, d, e2);
                Dout[(size_t)(b_ * 32 + i) * Jp + j] = o;
              }
            }
            if (zt_w) {  // the first sweep of a refinement block is z = A~^{-1} r, kept for the coupling sweeps
#pragma unroll
              for (int i = 0; i < 32; i++) Zt[(size_t)(b_ * 32 + i) * Jp + j] = __uint_as_float(r[i]);
            }
#pragma unroll
            for (int i = 0; i < 32; i++) dold[i] = dnxt[i];
          }
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tmem_empty)) : "memory");
        }
      }
      if (++kc == NKe) {
        kc = 0;
        it += gridDim.x;
        if (MIXED) {
          wi = wn;
          tile = wi.x;
        } else {
          tile += gridDim.x;
        }
      }
      if (++s == kBigStages) {
        s = 0;
        u3++;
      }
    }
  } else if (lane == 0) {
    // ------------------------------------------------ control: warp 8 issues the MMAs, warp 9 the copies
    const bool mma_role = w == kBigBuilders / 32;
    auto item_at = [&](int i_) { return items[(int)blockIdx.x + i_ * (int)gridDim.x]; };
    if (mma_role) {
      const uint32_t fmt = KIND == 1 ? 2u : 1u;  // kind::tf32 operands TF32 / kind::f16 operands BF16
      // instruction descriptor without N: F32 accumulator, both operands K-major, M = 128
      const uint32_t idesc0 = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kBigM >> 4) << 24);
      const uint64_t dhi = big_desc(0, 128, (uint32_t)(kBigKC * es / 16) * 128);  // descriptor without its address
      int n_m[kBigStages] = {0, 0, 0};
      for (int g = 0, s = 0, u3 = 0, kc = 0; g < n_chunks; g++) {
        // this chunk's RHS is built and its A^{-1} chunk has landed; a new tile waits for the drain
        bool ok = big_wait(su32(&rhs_full[s]), (uint32_t)(u3 & 1)) && big_wait(su32(&a_full[s]), (uint32_t)(u3 & 1));
        if (ok && kc == 0 && g > 0) ok = big_wait(su32(&tmem_empty), (uint32_t)(((g / NKe) - 1) & 1));
        if (!ok) {
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t bA = su32(sm + (size_t)s * stage_bytes);
        const uint32_t bR = bA + (uint32_t)(NT * kBigABlk);
        for (int nt = 0; nt < NT; nt++) {
          const int nn = min(kBigNT, n - nt * kBigNT);  // unknowns of this N-tile (a multiple of 16)
          const uint32_t idesc = idesc0 | ((uint32_t)(nn >> 3) << 17);
          const uint32_t d_tmem = tmem + (uint32_t)(nt * kBigNT);
          for (int pass = 0; pass < npass; pass++) {
            const uint32_t a0 = bR + (pass == 1 ? rpart : 0);                                 // RHS (cells x K)
            const uint32_t b0 = bA + (uint32_t)(nt * kBigABlk) + (pass == 2 ? apart : 0);  // A^{-1} rows (unknowns x K)
            for (int kk = 0; kk < ksteps; kk++) {
              const uint64_t ad = dhi | (uint64_t)(((a0 + kk * 256) & 0x3FFFF) >> 4);
              const uint64_t bd = dhi | (uint64_t)(((b0 + kk * 256) & 0x3FFFF) >> 4);
              const uint32_t acc = (kc > 0 || pass > 0 || kk > 0) ? 1u : 0u;
              if (KIND == 1)
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
                        d_tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
              else
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                        d_tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&mma_done[s])));
        n_m[s]++;
        if (++kc == NKe) kc = 0;
        if (++s == kBigStages) {
          s = 0;
          u3++;
        }
      }
      if (failed) {
        s_fail = 1;
        for (int q = 0; q < kBigStages; q++)  // MMAs still in flight finish before tensor memory is freed
          if (n_m[q] > 0) big_wait(su32(&mma_done[q]), (uint32_t)((n_m[q] - 1) & 1));
      }
    } else {
      int n_a[kBigStages] = {0, 0, 0}, n_in[kBigInBuf] = {0, 0, 0};
      // this CTA's work items, read ahead: icache[i & 3] is its i-th (tile, type) --
      // with one type per tile only the type, tau_of[i & 3], of its i-th tile
      int2 icache[4] = {make_int2(0, 0), make_int2(0, 0), make_int2(0, 0), make_int2(0, 0)};
      int tau_of[4] = {0, 0, 0, 0};
      auto tile_at = [&](int i_) { return (int)blockIdx.x + i_ * (int)gridDim.x; };
      for (int i = 0; i < 4 && i < my_items; i++) {
        if (MIXED) icache[i] = item_at(i);
        else tau_of[i] = type[tile_at(i) * kBigN];
      }
      int next_item = 4;  // the next item to read ahead
      auto issue_in = [&](int g_) {
        const int b_ = g_ % kBigInBuf;
        float *dst = (float *)(in_base + (size_t)b_ * kBigInBytes);
        const uint32_t bar = su32(&in_full[b_]);
        const int x0 = (MIXED ? icache[(g_ / NKe) & 3].x : tile_at(g_ / NKe)) * kBigN;
        const uint64_t tmd = reinterpret_cast<uint64_t>(dcur ? &tmD1 : &tmD0);
        if (half) {  // rows 32 kc .. 32 kc + 31 of the correction, as two boxes of 16
          const int y0 = (g_ % NKe) * 2 * kBigKC;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBigInHalf) : "memory");
          for (int h2 = 0; h2 < 2; h2++)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                    su32(dst + h2 * kBigKC * kBigDW)),
                "l"(tmd), "r"(x0 - kBigHalo), "r"(y0 + h2 * kBigKC), "r"(bar)
                : "memory");
        } else {
          const int y0 = (g_ % NKe) * kBigKC;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBigInFull) : "memory");
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                  su32(dst)),
              "l"(reinterpret_cast<uint64_t>(&tmR)), "r"(x0), "r"(y0), "r"(bar)
              : "memory");
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                  su32(dst + kBigKC * kBigN)),
              "l"(tmd), "r"(x0 - kBigHalo), "r"(y0), "r"(bar)
              : "memory");
        }
        n_in[b_]++;
      };
      auto issue_a = [&](int g_) {
        const int s_ = g_ % kBigStages;
        const int ti = g_ / NKe, tau_ = MIXED ? icache[ti & 3].y & 0x3FFFFFFF : tau_of[ti & 3], kc_ = g_ % NKe;
        unsigned char *dst = sm + (size_t)s_ * stage_bytes;
        const uint32_t bar = su32(&a_full[s_]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(NT * kBigABlk) : "memory");
        for (int nt = 0; nt < NT; nt++) {
          const unsigned char *src = (half ? AimgH : Aimg) + (((size_t)tau_ * NT + nt) * NKe + kc_) * kBigABlk;
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                           su32(dst + (size_t)nt * kBigABlk)),
                       "l"(reinterpret_cast<uint64_t>(src)), "r"(kBigABlk), "r"(bar)
                       : "memory");
        }
        n_a[s_]++;
      };
      for (int g = 0; g < kBigInBuf && g < n_chunks; g++) issue_in(g);
      for (int g = 0; g < kBigStages && g < n_chunks; g++) issue_a(g);
      for (int g = 0, s = 0, u3 = 0; g < n_chunks; g++) {
        // the builders have read chunk g's inputs: chunk g + 3's go into its buffer
        if (!big_wait(su32(&rhs_full[s]), (uint32_t)(u3 & 1))) {
          failed = true;
          break;
        }
        if (g + kBigInBuf < n_chunks) issue_in(g + kBigInBuf);
        // items up to three past the one whose chunk is issued now are read ahead: item i
        // takes the slot of item i - 4, all of whose copies have been issued (with one or
        // two chunks per item several items may become due in one step)
        for (const int due = (g + kBigStages) / NKe + 3; next_item < my_items && next_item <= due; next_item++) {
          if (MIXED) icache[next_item & 3] = item_at(next_item);
          else tau_of[next_item & 3] = type[tile_at(next_item) * kBigN];
        }
        // chunk g's MMAs are done: chunk g + 3's A^{-1} goes into its stage
        if (g + kBigStages < n_chunks) {
          if (!big_wait(su32(&mma_done[s]), (uint32_t)(u3 & 1))) {
            failed = true;
            break;
          }
          issue_a(g + kBigStages);
        }
        if (++s == kBigStages) {
          s = 0;
          u3++;
        }
      }
      if (failed) {
        s_fail = 1;
        // let the copies still in flight finish (bounded) before the CTA leaves
        for (int q = 0; q < kBigStages; q++)
          if (n_a[q] > 0) big_wait(su32(&a_full[q]), (uint32_t)((n_a[q] - 1) & 1));
        for (int q = 0; q < kBigInBuf; q++)
          if (n_in[q] > 0) big_wait(su32(&in_full[q]), (uint32_t)((n_in[q] - 1) & 1));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
  if (t == 0 && s_fail) {
    atomicExch(&ds->status, OCI_E_TIMEOUT);
    ds->done = 1;
  }
  double ve = (double)e2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ve += __shfl_down_sync(0xffffffffu, ve, o);
  if (lane == 0) red[w] = ve;
  __syncthreads();
  double bs = 0.0;
  if (t == 0)
    for (int i = 0; i < kBigThreads / 32; i++) bs += red[i];
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (t == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

static int tc_big_nt(const Handle &h) { return (4 * h.N * h.G + kBigNT - 1) / kBigNT; }
static int tc_big_nk(const Handle &h) { return (4 * h.N * h.G + kBigKC - 1) / kBigKC; }

size_t tc_big_smem(const Handle &h) {
  const size_t need = kBigStages * ((size_t)tc_big_nt(h) * kBigABlk + kBigRBlk) + kBigInBuf * (size_t)kBigInBytes + 1024;
  const size_t floor_bytes = 116 * 1024;  // one CTA per SM: its tensor memory never waits for another CTA's
  return need > floor_bytes ? need : floor_bytes;
}

// This kernel serves every size; OCI_TC_BIG=0 (a test hook) keeps the earlier
// persistent form with the inverse resident in shared memory (k_tc_pipe) for 4NG <= 128.
bool tc_big_used(const Handle &h) {
  if (4 * h.N * h.G > 128) return true;
  const char *e = hook_env("OCI_TC_BIG");
  return !(e && e[0] == '0');
}

int tc_big_prepare(Handle &h) {
  // tensor maps of r (z32) and of the two correction buffers, [R][Jp] FP32, boxes of
  // 32 rows x 128 cells (r) and 32 rows x 136 cells (the correction with its halo)
  typedef CUresult (*Encode)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  Encode enc = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t ee = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&enc, 12000, cudaEnableDefault, &q);
  if (ee != cudaSuccess || q != cudaDriverEntryPointSuccess || !enc)
    return set_error("cuTensorMapEncodeTiled is not available"), OCI_E_CUDA;
  const int R = 4 * h.N * h.G;
  const cuuint64_t dims[2] = {(cuuint64_t)h.Jp, (cuuint64_t)R};
  const cuuint64_t strides[1] = {(cuuint64_t)h.Jp * 4};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint32_t boxr[2] = {(cuuint32_t)kBigN, (cuuint32_t)kBigKC};
  const cuuint32_t boxd[2] = {(cuuint32_t)kBigDW, (cuuint32_t)kBigKC};
  CUresult r1 = enc(&h.tm_bg_r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.z32, dims, strides, boxr, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = enc(&h.tm_bg_d[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.delta[0], dims, strides, boxd, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r3 = enc(&h.tm_bg_d[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.delta[1], dims, strides, boxd, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS || r3 != CUDA_SUCCESS)
    return set_error("tensor maps of the tensor-core form could not be encoded"), OCI_E_CUDA;
  // work items: a tile of 128 cells per cell type present in it (in the order of first
  // appearance), so a region boundary inside a tile costs a second pass over that tile
  std::vector<int2> items;
  for (int t0 = 0; t0 < h.J; t0 += kBigN) {
    const int t1 = std::min(h.J, t0 + kBigN);
    std::vector<int> seen;
    for (int j = t0; j < t1; j++)
      if (std::find(seen.begin(), seen.end(), h.h_type[j]) == seen.end()) seen.push_back(h.h_type[j]);
    for (int tau : seen) items.push_back(make_int2(t0 / kBigN, tau | (seen.size() > 1 ? 0x40000000 : 0)));
  }
  if (h.tc_items) cudaFree(h.tc_items);
  h.tc_items = nullptr;
  cudaError_t ei = cudaMalloc(&h.tc_items, items.size() * sizeof(int2));
  if (ei == cudaSuccess)
    ei = cudaMemcpyAsync(h.tc_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, h.stream);
  if (ei == cudaSuccess) ei = cudaStreamSynchronize(h.stream);
  if (ei != cudaSuccess) return cuda_fail(ei, "tensor-core work items");
  h.tc_n_items = (int)items.size();
  h.tc_mixed = items.size() > (size_t)((h.J + kBigN - 1) / kBigN);
  const int sm = (int)tc_big_smem(h);
  cudaError_t e = cudaSuccess;
  for (const void *k : {(const void *)k_tc_big<1, false>, (const void *)k_tc_big<2, false>,
                        (const void *)k_tc_big<1, true>, (const void *)k_tc_big<2, true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_tc_big)");
  return OCI_OK;
}

int tc_big_grid(const Handle &h) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return h.tc_n_items < sms ? h.tc_n_items : sms;
}

void launch_tc_big(Handle &h, cudaGraphConditionalHandle cond, int use_cond) {
  const size_t smem = tc_big_smem(h);
  const int grid = tc_big_grid(h), NT = tc_big_nt(h), NK = tc_big_nk(h), NKH = 4 * h.N * h.G / 32;
#define OCI_TC_BIG_LAUNCH(K, M)                                                                                     \
  k_tc_big<K, M><<<grid, kBigThreads, smem, h.stream>>>(h.tm_bg_r, h.tm_bg_d[0], h.tm_bg_d[1], h.J, h.Jp, h.N, h.G, \
                                                        NT, NK, h.type, h.tc_img, h.mu32, h.z32, h.delta[0],          \
                                                        h.delta[1], h.ds, h.partials, h.counter, h.e_hist, cond,      \
                                                        use_cond, h.tc_items, h.tc_n_items, h.tc_img_h, NKH, h.tc_z)
  const bool tf = h.precision == OCI_TF32_IR;
  if (h.tc_mixed) {
    if (tf) OCI_TC_BIG_LAUNCH(1, true);
    else OCI_TC_BIG_LAUNCH(2, true);
  } else {
    if (tf) OCI_TC_BIG_LAUNCH(1, false);
    else OCI_TC_BIG_LAUNCH(2, false);
  }
#undef OCI_TC_BIG_LAUNCH
}

// Host: the per-type inverses in the chunk-major layout the kernel streams:
// block ((type * NT + nt) * NK + kc) holds rows 256 nt .. 256 nt + 255 (unknowns)
// and columns 16 kc .. 16 kc + 15 of A^{-1} (zero beyond n), TF32 -- or BF16 hi,
// then BF16 lo -- in the canonical K-major layout of big_off.  `round_tf32`,
// `bf16_bits` and `bf16_value` are the host roundings of the small form.
int tc_big_build_images(Handle &h, const std::vector<double> &Ainv, float (*round_tf32)(float),
                        uint16_t (*bf16_bits)(float), float (*bf16_value)(uint16_t)) {
  const int n = 4 * h.N * h.G, T = h.tt.n_types, NT = tc_big_nt(h), NK = tc_big_nk(h);
  const bool tf = h.precision == OCI_TF32_IR;
  const int es = tf ? 4 : 2;
  h.tc_img_bytes = (size_t)NT * NK * kBigABlk;
  std::vector<unsigned char> img((size_t)T * h.tc_img_bytes, 0);
  for (int t = 0; t < T; t++)
    for (int nt = 0; nt < NT; nt++)
      for (int kc = 0; kc < NK; kc++) {
        unsigned char *blk = img.data() + (((size_t)t * NT + nt) * NK + kc) * kBigABlk;
        for (int rl = 0; rl < kBigNT; rl++)
          for (int kl = 0; kl < kBigKC; kl++) {
            const int r = nt * kBigNT + rl, k = kc * kBigKC + kl;
            if (r >= n || k >= n) continue;
            const float v = (float)Ainv[((size_t)t * n + r) * n + k];
            const uint32_t off = big_off(rl, kl, es);
            if (tf) {
              const float q = round_tf32(v);
              memcpy(blk + off, &q, 4);
            } else {
              const uint16_t hi = bf16_bits(v);
              const uint16_t lo = bf16_bits(v - bf16_value(hi));
              memcpy(blk + off, &hi, 2);
              memcpy(blk + kBigABlk / 2 + off, &lo, 2);
            }
          }
      }
  cudaError_t e = cudaMalloc(&h.tc_img, img.size());
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tensor images)");
  e = cudaMemcpyAsync(h.tc_img, img.data(), img.size(), cudaMemcpyHostToDevice, h.stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(tensor images)");
  e = cudaStreamSynchronize(h.stream);
  if (e != cudaSuccess) return cuda_fail(e, "tensor images");
  // Coupling image, for n a multiple of 32: the inner sweeps after a refinement block's first are
  // delta = z + (A~^{-1} B) U, where B delta^i puts |mu_m| times an upstream corner
  // of the neighbour into two rows of each (group, angle) block -- kL, hL for mu > 0,
  // kR, hR for mu < 0 (Eq. rhs_sg applied to the correction).  Column 2 (gN + m) + s
  // (s = 0 time average, 1 time edge) of the image is |mu_m| times column
  // 4 (gN + m) + (mu_m > 0 ? 2s : 2s + 1) of A~^{-1}, laid out like the full image
  // with K = n / 2.  OCI_TC_HALF=0 (a test hook) keeps the full form for every sweep.
  const char *hv = hook_env("OCI_TC_HALF");
  if (n % 32 != 0 || (hv && hv[0] == '0')) return OCI_OK;
  const int NKH = n / 32, nh = n / 2;
  std::vector<unsigned char> imh((size_t)T * NT * NKH * kBigABlk, 0);
  for (int t = 0; t < T; t++)
    for (int nt = 0; nt < NT; nt++)
      for (int kc = 0; kc < NKH; kc++) {
        unsigned char *blk = imh.data() + (((size_t)t * NT + nt) * NKH + kc) * kBigABlk;
        for (int rl = 0; rl < kBigNT; rl++)
          for (int kl = 0; kl < kBigKC; kl++) {
            const int r = nt * kBigNT + rl, k = kc * kBigKC + kl;
            if (r >= n || k >= nh) continue;
            const int gm = k / 2, sc = k % 2, m = gm % h.N;
            const bool pos = m >= h.N / 2;
            const int col = 4 * gm + (pos ? 2 * sc : 2 * sc + 1);
            const float v = (float)(fabs(h.h_mu[m]) * Ainv[((size_t)t * n + r) * n + col]);
            const uint32_t off = big_off(rl, kl, es);
            if (tf) {
              const float q = round_tf32(v);
              memcpy(blk + off, &q, 4);
            } else {
              const uint16_t hi = bf16_bits(v);
              const uint16_t lo = bf16_bits(v - bf16_value(hi));
              memcpy(blk + off, &hi, 2);
              memcpy(blk + kBigABlk / 2 + off, &lo, 2);
            }
          }
      }
  e = cudaMalloc(&h.tc_img_h, imh.size());
  if (e == cudaSuccess) e = cudaMalloc(&h.tc_z, (size_t)n * h.Jp * sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(h.tc_z, 0, (size_t)n * h.Jp * sizeof(float), h.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.tc_img_h, imh.data(), imh.size(), cudaMemcpyHostToDevice, h.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h.stream);
  if (e != cudaSuccess) return cuda_fail(e, "tensor coupling image");
  return OCI_OK;
}

}  // namespace oci
