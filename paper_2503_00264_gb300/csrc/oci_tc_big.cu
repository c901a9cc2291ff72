// oci_tc_big.cu -- tcgen05 block apply of the TF32 / BF16x3 mixed forms for cells
// with more than 128 unknowns (128 < 4NG <= 512, e.g. S16 with 8 groups).
//
// The inner sweep of the mixed forms is delta^{i+1} = A~^{-1} (r + B delta^i) per
// cell (spec: where cells share material, width and dt, the inverse of
// the cell matrix of Eqs. Aj, scatter, fullOCIlhs is applied to all of their
// right-hand sides as one dense GEMM).  For a tile of 128 cells of one type this
// is, transposed so that the cells are the MMA's M and the unknowns its N,
//   D[128 cells x n] = RHS[128 cells x n] . (A^{-1})^T,      n = 4NG <= 512,
// with the accumulator in tensor memory (lane = cell, column = unknown; n
// columns).  The inverse (1 MB per type in TF32) does not fit in shared memory:
//   - the K dimension is walked in chunks of 32: per chunk one 1D bulk copy per
//     N-tile of 256 unknowns brings that chunk of A^{-1} (32 KB, stored chunk
//     by chunk in the K-major no-swizzle canonical layout) into shared memory,
//     and two 2D tensor copies bring rows k .. k+31 of r and of the old
//     correction (with a halo of 4 cells each side for the neighbours' inflow);
//     all threads then build that chunk of the RHS (r + B delta, FP32 -> TF32 or
//     BF16 hi/lo) next to it;
//   - the MMAs of a chunk (M = 128 cells, N = 256 unknowns, one thread issues
//     them, completion on an mbarrier) read the RHS chunk once per N-tile and
//     each A^{-1} row once;
//   - two stages: the MMAs of chunk k run while the copies and the RHS of chunk
//     k+1 are prepared; the copies of chunk k+1 start as soon as chunk k-1's
//     MMAs free their stage;
//   - after the last chunk of a tile the CTA drains the accumulators
//     (tcgen05.ld: one register per unknown, one lane per cell), forms delta
//     and the FP32 norm partial; loads and stores are 128-byte rows of 32 cells.
// One CTA per SM walks the tiles persistently; the norm, the stop rule and the
// refinement decision are fused into the last CTA to finish.  Every wait is
// bounded: on a timeout the CTA waits (bounded) for its copies and MMAs in
// flight, frees its tensor memory and records OCI_E_TIMEOUT.
#include <cuda_bf16.h>
#include <math.h>

#include <vector>

#include "oci_device.cuh"
#include "oci_internal.h"

namespace oci {

constexpr int kBigM = 128;        // MMA M: cells per tile
constexpr int kBigN = 128;        // cells per tile (the M of the MMA)
constexpr int kBigNT = 256;       // MMA N: unknowns per N-tile
constexpr int kBigKC = 32;        // K elements per chunk
constexpr int kBigABlk = 32768;   // one chunk of A^{-1} for one N-tile: 256 rows x 32 K (TF32, or BF16 hi + lo)
constexpr int kBigRBlk = 16384;   // one chunk of the RHS: 128 cells x 32 K (TF32, or BF16 hi + lo)
constexpr int kBigThreads = 256;
constexpr long long kBigSpin = 1 << 22;
constexpr int kBigHalo = 4;                       // columns each side of the delta box (16 B)
constexpr int kBigDW = kBigN + 2 * kBigHalo;      // delta box width
constexpr int kBigInBytes = kBigKC * (kBigN + kBigDW) * 4;  // r box + delta box of one chunk

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

template <int KIND>  // 1 = TF32, 2 = BF16 x3
__global__ void __launch_bounds__(kBigThreads, 1) k_tc_big(
    const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmD0,
    const __grid_constant__ CUtensorMap tmD1, int J, int Jp, int N, int G, int NT, int NK, const int32_t *__restrict__ type,
    const unsigned char *__restrict__ Aimg, const float *__restrict__ mu, const float *__restrict__ r32, float *D0,
    float *D1, DevState *ds, double *__restrict__ partials, unsigned *counter, double *e_hist,
    cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(1024) unsigned char smb_[];
  __shared__ __align__(8) uint64_t tma_bar[2], mma_bar[2], in_bar;
  __shared__ uint32_t tslot;
  __shared__ double red[kBigThreads / 32];
  __shared__ bool s_last;
  __shared__ int s_fail;
  constexpr int es = KIND == 1 ? 4 : 2;
  constexpr int apart = kBigABlk / 2;  // BF16: the lo image follows the hi image
  constexpr int rpart = kBigRBlk / 2;
  const int n = 4 * N * G;
  unsigned char *sm = (unsigned char *)(((uintptr_t)smb_ + 1023) & ~(uintptr_t)1023);
  const size_t stage_bytes = (size_t)NT * kBigABlk + kBigRBlk;  // NT A^{-1} blocks, then the RHS block
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (ds->done) return;  // uniform
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  const uint32_t cols = n <= 256 ? 256u : 512u;  // one column per unknown
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    for (int s = 0; s < 2; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&tma_bar[s])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mma_bar[s])), "r"(1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&in_bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const int ntiles = (J + kBigN - 1) / kBigN;
  const int N2 = N / 2;
  const uint32_t fmt = KIND == 1 ? 2u : 1u;  // kind::tf32 operands TF32 / kind::f16 operands BF16
  // instruction descriptor without N: F32 accumulator, both operands K-major, M = 128
  const uint32_t idesc0 = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kBigM >> 4) << 24);
  const uint32_t lbo = 128, sbo = (uint32_t)(kBigKC * es / 16) * 128;
  constexpr int ksteps = kBigKC * es / 32;  // MMAs per chunk and pass (K = 8 TF32 / 16 BF16)
  constexpr int npass = KIND == 1 ? 1 : 3;  // BF16 x3: hi.hi + hi.lo + lo.hi
  // per-stage counts kept by thread 0 (copies issued, MMA groups committed)
  int n_tma[2] = {0, 0}, n_mma[2] = {0, 0}, n_in = 0;
  float e2 = 0.f;
  bool failed = false;
  // RHS inputs of a chunk, staged by the tensor memory accelerator into one
  // buffer after the two stages: rows kb .. kb+31 of r (128 cells) and of the old
  // correction (cells j0-4 .. j0+131, the halo for the neighbours' inflow; a box
  // reaching past the array reads zeros).  Thread t owns cell c = t % 128 and
  // the 16 rows hh*16 .. hh*16+15 of the chunk.
  const int c = t & (kBigN - 1), hh = t >> 7;
  float *in_r = (float *)(sm + 2 * stage_bytes);  // [32][128]
  float *in_d = in_r + kBigKC * kBigN;            // [32][136]
  const CUtensorMap *tmD = dcur ? &tmD1 : &tmD0;
  auto issue_in = [&](int tile_, int kc_) {  // thread 0
    const uint32_t bar = su32(&in_bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBigInBytes) : "memory");
    const int x0 = tile_ * kBigN, y0 = kc_ * kBigKC;
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(in_r)),
        "l"(reinterpret_cast<uint64_t>(&tmR)), "r"(x0), "r"(y0), "r"(bar)
        : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(in_d)),
        "l"(reinterpret_cast<uint64_t>(tmD)), "r"(x0 - kBigHalo), "r"(y0), "r"(bar)
        : "memory");
    n_in++;
  };
  // the A copies of chunk gk_ (type tau_, chunk kc_) into stage gk_ & 1; thread 0
  auto issue_tma = [&](int gk_, int tau_, int kc_) {
    const int s_ = gk_ & 1;
    const uint32_t bar = su32(&tma_bar[s_]);
    unsigned char *stA_ = sm + (size_t)s_ * stage_bytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(NT * kBigABlk) : "memory");
    for (int nt = 0; nt < NT; nt++) {
      const unsigned char *src = Aimg + (((size_t)tau_ * NT + nt) * NK + kc_) * kBigABlk;
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       su32(stA_ + (size_t)nt * kBigABlk)),
                   "l"(reinterpret_cast<uint64_t>(src)), "r"(kBigABlk), "r"(bar)
                   : "memory");
    }
    n_tma[s_]++;
  };
  auto advance = [&](int &tl, int &k) {
    if (++k == NK) {
      k = 0;
      tl += gridDim.x;
    }
  };
  const uint64_t dhi = big_desc(0, lbo, sbo);  // descriptor without its start address
  int tile = blockIdx.x, kc = 0, gk = 0;
  int tau_cur = 0, tau_nt = 0;  // types of the current and the next tile (thread 0)
  // one chunk: returns 0 to go on, 1 when this CTA's work is done, -1 on a failure
  auto chunk = [&]() -> int {
    const int s = gk & 1;
    unsigned char *stA = sm + (size_t)s * stage_bytes;
    unsigned char *stB = stA + (size_t)NT * kBigABlk;  // the RHS chunk: the MMA's A operand
    int ntile = tile, nkc = kc;
    advance(ntile, nkc);
    const bool has_next = ntile < ntiles;
    // (1) stage s is free once the MMAs of chunk gk - 2 have completed, and this
    // chunk's inputs have landed: thread 0 waits on the mbarriers (acquire), the
    // others in the block barrier behind it
    bool ok = true;
    if (t == 0) {
      if (gk >= 2) ok = big_wait(su32(&mma_bar[s]), (uint32_t)(((gk >> 1) - 1) & 1));
      ok = ok && big_wait(su32(&in_bar), (uint32_t)(gk & 1));
    }
    if (!__syncthreads_and(ok && s_fail == 0)) return -1;
    // (2) this chunk's RHS r + B delta into the stage: TF32 or BF16 hi/lo
    {
      const int j = tile * kBigN + c;
      const bool act = j < J;
      const int kb = kc * kBigKC + hh * 16;
      float vc[16];
#pragma unroll
      for (int i = 0; i < 16; i++) vc[i] = act ? in_r[(hh * 16 + i) * kBigN + c] : 0.f;
      if (act && !zero) {
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int k = kb + 2 * q, kl2 = hh * 16 + 2 * q;
          const int m = (k >> 2) % N;
          const float mf = mu[m];
          if (m >= N2) {  // p even: mu * (R corner of cell j-1)
            if (j > 0) vc[2 * q] = fmaf(mf, in_d[(kl2 + 1) * kBigDW + c + kBigHalo - 1], vc[2 * q]);
          } else if (j < J - 1) {  // p odd: |mu| * (L corner of cell j+1)
            vc[2 * q + 1] = fmaf(-mf, in_d[kl2 * kBigDW + c + kBigHalo + 1], vc[2 * q + 1]);
          }
        }
      }
      const int kl = hh * 16;  // row inside the chunk
      if (KIND == 1) {
#pragma unroll
        for (int g4 = 0; g4 < 16; g4 += 4)
          *(float4 *)(stB + big_off(c, kl + g4, 4)) = make_float4(vc[g4], vc[g4 + 1], vc[g4 + 2], vc[g4 + 3]);
      } else {
#pragma unroll
        for (int g8 = 0; g8 < 16; g8 += 8) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const float a0 = vc[g8 + 2 * i], a1 = vc[g8 + 2 * i + 1];
            const __nv_bfloat16 h0 = __float2bfloat16_rn(a0), h1 = __float2bfloat16_rn(a1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(a0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(a1 - __bfloat162float(h1));
            hi[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lo[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
          }
          const uint32_t off = big_off(c, kl + g8, 2);
          *(uint4 *)(stB + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *(uint4 *)(stB + rpart + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
    }
    // (4) the RHS is visible to the tensor cores; the previous tile's drain is done
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // (5) one thread: wait for this chunk's copies, issue the MMAs of every M-tile and
    // commit; then, once chunk gk - 1's MMAs have freed the other stage, start the
    // copies of chunk gk + 1 into it
    if (t == 0) {
      if (has_next) issue_in(ntile, nkc);  // every thread has read this chunk's inputs
      if (!big_wait(su32(&tma_bar[s]), (uint32_t)((gk >> 1) & 1))) {
        s_fail = 1;
      } else {
        const uint32_t bA = su32(stA), bR = su32(stB);
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
            su32(&mma_bar[s])));
        n_mma[s]++;
        if (has_next) {
          if (gk >= 1 && !big_wait(su32(&mma_bar[s ^ 1]), (uint32_t)(((gk - 1) >> 1) & 1))) s_fail = 1;
          else issue_tma(gk + 1, nkc == 0 ? tau_nt : tau_cur, nkc);
        }
      }
    }
    // (6) last chunk of the tile: drain the accumulators.  Warp w reads the lanes
    // (cells) 32 (w % 4) .. +31; the n columns (unknowns) go in blocks of 32 to
    // the two warps of a lane quarter alternately; each register of a block is one
    // unknown of the lane's cell, so every load and store is a 128-byte row of 32
    // cells.  The old correction of the next block is loaded before this one's
    // accumulators are read.
    if (kc == NK - 1) {
      bool okd = true;
      if (t == 0) okd = s_fail == 0 && big_wait(su32(&mma_bar[s]), (uint32_t)((gk >> 1) & 1));
      if (!__syncthreads_and(okd)) return -1;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int q4 = w & 3, g2 = w >> 2;
      const int j = tile * kBigN + 32 * q4 + lane;
      const bool act = j < J;
      const int nb = n / 32;  // column blocks
      float dold[32], dnxt[32];
      auto load_old = [&](int b_, float *dst) {
#pragma unroll
        for (int i = 0; i < 32; i++) dst[i] = (act && !zero) ? Din[(size_t)(b_ * 32 + i) * Jp + j] : 0.f;
      };
      if (g2 < nb) load_old(g2, dold);
#pragma unroll 1
      for (int b_ = g2; b_ < nb; b_ += 2) {
        uint32_t r[32];
        const uint32_t addr = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(b_ * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
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
#pragma unroll
        for (int i = 0; i < 32; i++) dold[i] = dnxt[i];
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if (t == 0 && nkc == 0 && has_next) {  // entering the next tile: its type, and the one after
      tau_cur = tau_nt;
      if (ntile + (int)gridDim.x < ntiles) tau_nt = type[(ntile + gridDim.x) * kBigN];
    }
    tile = ntile;
    kc = nkc;
    gk++;
    return has_next ? 0 : 1;
  };
  if (tile < ntiles) {
    if (t == 0) {
      tau_cur = type[tile * kBigN];
      if (tile + (int)gridDim.x < ntiles) tau_nt = type[(tile + gridDim.x) * kBigN];
      issue_in(tile, 0);
      issue_tma(0, tau_cur, 0);
    }
    for (;;) {
      const int rc = chunk();
      if (rc != 0) {
        failed = rc < 0;
        break;
      }
    }
  }
  if (failed && t == 0) {
    // let the copies and MMAs still in flight finish (bounded) before tensor memory is freed
    for (int s = 0; s < 2; s++) {
      if (n_tma[s] > 0) big_wait(su32(&tma_bar[s]), (uint32_t)((n_tma[s] - 1) & 1));
      if (n_mma[s] > 0) big_wait(su32(&mma_bar[s]), (uint32_t)((n_mma[s] - 1) & 1));
    }
    if (n_in > 0) big_wait(su32(&in_bar), (uint32_t)((n_in - 1) & 1));
    atomicExch(&ds->status, OCI_E_TIMEOUT);
    ds->done = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
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
  const size_t need = 2 * ((size_t)tc_big_nt(h) * kBigABlk + kBigRBlk) + kBigInBytes + 1024;
  const size_t floor_bytes = 116 * 1024;  // one CTA per SM: its tensor memory never waits for another CTA's
  return need > floor_bytes ? need : floor_bytes;
}

bool tc_big_used(const Handle &h) { return 4 * h.N * h.G > 128; }

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
  const int sm = (int)tc_big_smem(h);
  cudaError_t e = cudaFuncSetAttribute(k_tc_big<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_big<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_tc_big)");
  return OCI_OK;
}

int tc_big_grid(const Handle &h) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = (h.J + kBigN - 1) / kBigN;
  return ntiles < sms ? ntiles : sms;
}

void launch_tc_big(Handle &h, cudaGraphConditionalHandle cond, int use_cond) {
  const size_t smem = tc_big_smem(h);
  const int grid = tc_big_grid(h), NT = tc_big_nt(h), NK = tc_big_nk(h);
  if (h.precision == OCI_TF32_IR)
    k_tc_big<1><<<grid, kBigThreads, smem, h.stream>>>(h.tm_bg_r, h.tm_bg_d[0], h.tm_bg_d[1], h.J, h.Jp, h.N, h.G, NT, NK, h.type, h.tc_img, h.mu32, h.z32,
                                                        h.delta[0], h.delta[1], h.ds, h.partials, h.counter,
                                                        h.e_hist, cond, use_cond);
  else
    k_tc_big<2><<<grid, kBigThreads, smem, h.stream>>>(h.tm_bg_r, h.tm_bg_d[0], h.tm_bg_d[1], h.J, h.Jp, h.N, h.G, NT, NK, h.type, h.tc_img, h.mu32, h.z32,
                                                        h.delta[0], h.delta[1], h.ds, h.partials, h.counter,
                                                        h.e_hist, cond, use_cond);
}

// Host: the per-type inverses in the chunk-major layout the kernel streams:
// block ((type * NT + nt) * NK + kc) holds rows 256 nt .. 256 nt + 255 (unknowns)
// and columns 32 kc .. 32 kc + 31 of A^{-1} (zero beyond n), TF32 -- or BF16 hi,
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
  return OCI_OK;
}

}  // namespace oci
