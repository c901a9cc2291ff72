// oci_tc.cu -- tensor-core (tcgen05) block apply of the mixed-precision form.
//
// For cells that share (material, dx, dt) the inverse of the dense cell matrix
// A = L_c - S (order n = 4NG, Eqs. Aja, Aj, scatter, fullOCIlhs) is one matrix;
// the inner sweep of the mixed form,
//     delta^{i+1}_j = A^{-1} (r_j + B delta^i),
// is then a GEMM  D[n x 128 cells] = A^{-1}[n x n] * RHS[n x 128 cells]  per tile
// of 128 cells.  It runs on the 5th-generation tensor cores:
//   - A^{-1} (rows padded to M = 128) is stored once per type, pre-arranged in
//     the K-major no-swizzle canonical layout (8-row x 16-byte core matrices),
//     and copied into shared memory;
//   - the RHS tile r + B delta is formed in FP32 by the CTA and written in the
//     same layout (TF32, or BF16 hi/lo for the 3-product split);
//   - one thread issues tcgen05.mma (kind::tf32, or kind::f16 with BF16 inputs:
//     A_hi B_hi + A_hi B_lo + A_lo B_hi) accumulating in FP32 in tensor memory;
//     completion is signalled through an mbarrier (bounded wait);
//   - tcgen05.ld moves D to registers, a shared-memory transpose makes the
//     stores coalesced, and the FP64-accumulated norm partial is written.
// Requires n <= 128, n % 32 == 0, and one cell type per aligned 128-cell tile.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "oci_device.cuh"

namespace oci {

constexpr int kTcM = 128;   // MMA M (rows of A^{-1}, padded)
constexpr int kTcN = 128;   // MMA N (cells per tile)
constexpr int kTcCols = 128;  // TMEM columns allocated (FP32 accumulator, N columns)
constexpr long long kTcSpin = 1 << 22;

// Bounded wait for phase `parity` of an mbarrier in shared memory.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok = 0;
  for (long long it = 0; it < kTcSpin && !ok; it++) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (!ok) __nanosleep(32);
  }
  return ok != 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, no swizzle
}

// byte offset of (row, k) in the K-major no-swizzle layout of a [rows x K] operand
__host__ __device__ inline uint32_t kmajor_off(int row, int k, int es, int kbytes) {
  const int kc = 16 / es;
  return (uint32_t)((row / 8) * (kbytes / 16) * 128 + (k / kc) * 128 + (row % 8) * 16 + (k % kc) * es);
}

template <int KIND>  // 1 = TF32, 2 = BF16 x3
__global__ void __launch_bounds__(128) k_tc_inner(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                                                  const unsigned char *__restrict__ Aimg, size_t a_bytes_per_type,
                                                  const double *__restrict__ mu, const float *__restrict__ r32,
                                                  float *D0, float *D1, DevState *ds,
                                                  double *__restrict__ partials) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ double red[4];
  const int n = 4 * N * G;
  constexpr int es = KIND == 1 ? 4 : 2;
  const int kbytes = n * es;
  const int opb = kTcM * kbytes;   // bytes of one operand image (A or B, one part)
  constexpr int parts = KIND == 1 ? 1 : 2;
  unsigned char *sA = sm;                 // parts x opb
  unsigned char *sB = sm + parts * opb;   // parts x opb
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (ds->done) return;  // uniform
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  const int j0 = blockIdx.x * kTcN;
  const int tau = type[j0];

  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // A^{-1} image of this type (already in the canonical layout)
  {
    const uint4 *src = (const uint4 *)(Aimg + (size_t)tau * a_bytes_per_type);
    uint4 *dst = (uint4 *)sA;
    const int nv = parts * opb / 16;
    for (int i = t; i < nv; i += 128) dst[i] = src[i];
  }
  // RHS tile: thread t owns cell j = j0 + t (row t of the N x K operand).
  // Eight independent loads are issued before any is used (memory-level parallelism).
  {
    const int j = j0 + t;
    const bool act = j < J;
    const int N2 = N / 2;
    for (int k0 = 0; k0 < n; k0 += 8) {
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; i++) v[i] = act ? r32[(size_t)(k0 + i) * Jp + j] : 0.f;
      if (act && !zero) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const int k = k0 + i;
          const int gm = k >> 2, p = k & 3, m = gm % N;
          if (m >= N2) {
            if ((p == 0 || p == 2) && j > 0) v[i] = fmaf((float)mu[m], Din[(size_t)(k + 1) * Jp + j - 1], v[i]);
          } else {
            if ((p == 1 || p == 3) && j < J - 1) v[i] = fmaf(-(float)mu[m], Din[(size_t)(k - 1) * Jp + j + 1], v[i]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const uint32_t off = kmajor_off(t, k0 + i, es, kbytes);
        if (KIND == 1) {
          *(float *)(sB + off) = v[i];
        } else {
          const __nv_bfloat16 hi = __float2bfloat16_rn(v[i]);
          const __nv_bfloat16 lo = __float2bfloat16_rn(v[i] - __bfloat162float(hi));
          *(__nv_bfloat16 *)(sB + off) = hi;
          *(__nv_bfloat16 *)(sB + opb + off) = lo;
        }
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  if (t == 0) {
    const uint32_t fmt = KIND == 1 ? 2u : 1u;  // TF32 (kind::tf32) / BF16 (kind::f16)
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);
    const uint32_t lbo = 128, sbo = (uint32_t)(kbytes / 16) * 128;
    const int ksteps = kbytes / 32;  // 32 bytes of K per instruction
    const int npass = KIND == 1 ? 1 : 3;
    int issued = 0;
    for (int pass = 0; pass < npass; pass++) {
      // pass 0: A_hi B_hi, pass 1: A_hi B_lo, pass 2: A_lo B_hi
      const uint32_t a0 = smem_u32(sA) + (pass == 2 ? opb : 0);
      const uint32_t b0 = smem_u32(sB) + (pass == 1 ? opb : 0);
      for (int kk = 0; kk < ksteps; kk++, issued++) {
        const uint64_t ad = tc_desc(a0 + kk * 256, lbo, sbo);
        const uint64_t bd = tc_desc(b0 + kk * 256, lbo, sbo);
        const uint32_t acc = issued > 0 ? 1u : 0u;
        if (KIND == 1)
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                       "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        else
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                       "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
  }
  uint32_t ok = 0;
  for (long long it = 0; it < kTcSpin && !ok; it++) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(&mbar)), "r"(0));
    if (!ok) __nanosleep(32);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  // D (rows = unknowns, columns = cells) -> shared memory [n][129] for coalesced stores
  float *Dt = (float *)sm;  // aliases the operand images (no longer read by the MMA)
  __syncthreads();
  if (ok) {
    const int row = 32 * w + lane;
    for (int c0 = 0; c0 < kTcN; c0 += 32) {
      uint32_t r[32];
      const uint32_t addr = tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < n)
#pragma unroll
        for (int i = 0; i < 32; i++) Dt[row * (kTcN + 1) + c0 + i] = __uint_as_float(r[i]);
    }
  } else if (t == 0) {
    // one more bounded wait: the MMA issued above may still read the operand
    // images and write the accumulator that is freed below
    tc_wait(smem_u32(&mbar), 0);
    atomicExch(&ds->status, OCI_E_TIMEOUT);
    ds->done = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
  double e2 = 0.0;
  if (ok) {
    const int j = j0 + t;
    if (j < J) {
      float acc = 0.f;
      for (int k0 = 0; k0 < n; k0 += 8) {
        float old[8];
#pragma unroll
        for (int i = 0; i < 8; i++) old[i] = zero ? 0.f : Din[(size_t)(k0 + i) * Jp + j];
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const float o = Dt[(k0 + i) * (kTcN + 1) + t];
          const float d = o - old[i];
          acc = fmaf(d, d, acc);
          Dout[(size_t)(k0 + i) * Jp + j] = o;
        }
      }
      e2 = (double)acc;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, o);
  if (lane == 0) red[w] = e2;
  __syncthreads();
  if (t == 0) partials[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

size_t tc_smem(const Handle &h) {
  const int n = 4 * h.N * h.G;
  const int es = h.precision == OCI_TF32_IR ? 4 : 2;
  const int parts = h.precision == OCI_TF32_IR ? 1 : 2;
  size_t ops = (size_t)2 * parts * kTcM * n * es;
  size_t dt = (size_t)n * (kTcN + 1) * 4;
  return (ops > dt ? ops : dt) + 1024;
}

int tc_partials(const Handle &h) { return (h.J + kTcN - 1) / kTcN; }

void launch_tc_inner(Handle &h) {
  const size_t smem = tc_smem(h);
  if (h.precision == OCI_TF32_IR)
    k_tc_inner<1><<<tc_partials(h), 128, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tc_img, h.tc_img_bytes, h.mu,
                                                           h.z32, h.delta[0], h.delta[1], h.ds, h.partials);
  else
    k_tc_inner<2><<<tc_partials(h), 128, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tc_img, h.tc_img_bytes, h.mu,
                                                           h.z32, h.delta[0], h.delta[1], h.ds, h.partials);
}


// ---------------------------------------------------------------- persistent, pipelined form
// One CTA per SM walks the tiles tile = blockIdx.x, blockIdx.x + gridDim.x, ...
// with all the types' A^{-1} images resident in shared memory (loaded once),
// the RHS operand double-buffered in shared memory and two 128-column FP32
// accumulators in tensor memory: while the tensor cores run tile i (issued by
// one thread, completion on an mbarrier), the CTA drains tile i-1 from TMEM
// (tcgen05.ld straight into registers, vectorised stores of delta and the
// norm) and builds the RHS of tile i+1.  The norm, stop rule and refinement
// decision are fused into the last CTA.  Every wait is bounded; on a timeout
// the kernel waits (bounded) for its MMAs in flight, frees TMEM and records
// OCI_E_TIMEOUT.
constexpr int kTcPipeThreads = 256;


// KB rows k0..k0+KB-1 of one cell's RHS r + B delta (FP32), written into the
// K-major operand image (TF32, or BF16 hi/lo); all loads first.
template <int KIND, int KB>
__device__ __forceinline__ void tc_rhs_rows(int k0, int c, int j, bool act, bool zero, int J, int Jp, int N, int N2,
                                            int kbytes, int opb, const float *__restrict__ mu,
                                            const float *__restrict__ r32, const float *__restrict__ Din,
                                            unsigned char *b) {
  float v[KB], u[KB / 2];
#pragma unroll
  for (int i = 0; i < KB; i++) v[i] = act ? r32[(size_t)(k0 + i) * Jp + j] : 0.f;
  // rows p = 0, 2 (mu > 0) take the R corner of cell j-1; rows p = 1, 3 (mu < 0)
  // the L corner of cell j+1: one inflow value per row pair
#pragma unroll
  for (int q = 0; q < KB / 2; q++) {
    const int i = 2 * q;  // rows k0+i (p even) and k0+i+1 (p odd)
    const int k = k0 + i;
    const int m = (k >> 2) % N;
    u[q] = 0.f;
    if (act && !zero) {
      if (m >= N2) {
        if (j > 0) u[q] = Din[(size_t)(k + 1) * Jp + j - 1];
      } else if (j < J - 1) {
        u[q] = Din[(size_t)k * Jp + j + 1];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < KB / 2; q++) {
    const int k = k0 + 2 * q;
    const int m = (k >> 2) % N;
    const float mf = mu[m];
    if (m >= N2) v[2 * q] = fmaf(mf, u[q], v[2 * q]);  // p even gets mu * psi_{j-1}(p+1)
    else v[2 * q + 1] = fmaf(-mf, u[q], v[2 * q + 1]);  // p odd gets |mu| * psi_{j+1}(p-1)
  }
#pragma unroll
  for (int g8 = 0; g8 < KB; g8 += 8) {
    if (KIND == 1) {
      *(float4 *)(b + kmajor_off(c, k0 + g8, 4, kbytes)) = make_float4(v[g8], v[g8 + 1], v[g8 + 2], v[g8 + 3]);
      *(float4 *)(b + kmajor_off(c, k0 + g8 + 4, 4, kbytes)) =
          make_float4(v[g8 + 4], v[g8 + 5], v[g8 + 6], v[g8 + 7]);
    } else {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const float a0 = v[g8 + 2 * i], a1 = v[g8 + 2 * i + 1];
        const __nv_bfloat16 h0 = __float2bfloat16_rn(a0), h1 = __float2bfloat16_rn(a1);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(a0 - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(a1 - __bfloat162float(h1));
        hi[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        lo[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
      }
      const uint32_t off = kmajor_off(c, k0 + g8, 2, kbytes);
      *(uint4 *)(b + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *(uint4 *)(b + opb + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(kTcPipeThreads, 1) k_tc_pipe(
    int J, int Jp, int N, int G, int n_types, const int32_t *__restrict__ type, const unsigned char *__restrict__ Aimg,
    const float *__restrict__ mu, const float *__restrict__ r32, float *D0, float *D1, DevState *ds,
    double *__restrict__ partials, unsigned *counter, double *e_hist, cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(1024) unsigned char smt_[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  __shared__ double red[8];
  __shared__ bool s_last;
  const int n = 4 * N * G;
  constexpr int es = KIND == 1 ? 4 : 2;
  constexpr int parts = KIND == 1 ? 1 : 2;
  const int kbytes = n * es;
  const int opb = kTcM * kbytes;
  unsigned char *sm = (unsigned char *)(((uintptr_t)smt_ + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = sm;                                    // [type][part][opb]
  unsigned char *sB = sA + (size_t)n_types * parts * opb;  // [stage][part][opb]
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int nthr = kTcPipeThreads;
  if (ds->done) return;  // uniform
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(2 * kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  {
    const uint4 *src = (const uint4 *)Aimg;
    uint4 *dst = (uint4 *)sA;
    const int nv = n_types * parts * opb / 16;
    for (int i = t; i < nv; i += nthr) dst[i] = src[i];
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const int ntiles = (J + kTcN - 1) / kTcN;
  const int N2 = N / 2;
  const uint32_t fmt = KIND == 1 ? 2u : 1u;
  const uint32_t idesc =
      (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  const uint32_t lbo = 128, sbo = (uint32_t)(kbytes / 16) * 128;
  float e2 = 0.f;
  int it = 0, prev = -1;
  bool failed = false;
  for (int tile = blockIdx.x;; tile += gridDim.x, it++) {
    const bool have = tile < ntiles;
    const int st = it & 1;
    if (have) {
      // RHS of this tile: thread t builds cell c = t % 128, rows [h*n/2, (h+1)*n/2),
      // in batches whose loads are all issued before any is used
      const int c = t & (kTcN - 1), hh = t >> 7;
      const int j = tile * kTcN + c;
      const bool act = j < J;
      unsigned char *b = sB + (size_t)st * parts * opb;
      const int kh = n / 2;
      if (kh % 32 == 0)
        for (int k0 = hh * kh; k0 < (hh + 1) * kh; k0 += 32)
          tc_rhs_rows<KIND, 32>(k0, c, j, act, zero, J, Jp, N, N2, kbytes, opb, mu, r32, Din, b);
      else
        for (int k0 = hh * kh; k0 < (hh + 1) * kh; k0 += 16)
          tc_rhs_rows<KIND, 16>(k0, c, j, act, zero, J, Jp, N, N2, kbytes, opb, mu, r32, Din, b);
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (t == 0) {
        const int tau = type[tile * kTcN];
        const unsigned char *a = sA + (size_t)tau * parts * opb;
        const uint32_t d_tmem = tmem + (uint32_t)(st * kTcCols);
        const int ksteps = kbytes / 32;
        const int npass = KIND == 1 ? 1 : 3;
        int issued = 0;
        for (int pass = 0; pass < npass; pass++) {
          const uint32_t a0 = smem_u32(a) + (pass == 2 ? opb : 0);
          const uint32_t b0 = smem_u32(b) + (pass == 1 ? opb : 0);
          for (int kk = 0; kk < ksteps; kk++, issued++) {
            const uint64_t ad = tc_desc(a0 + kk * 256, lbo, sbo);
            const uint64_t bd = tc_desc(b0 + kk * 256, lbo, sbo);
            const uint32_t acc = issued > 0 ? 1u : 0u;
            if (KIND == 1)
              asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
                           "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            else
              asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
                           "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&mbar[st])));
      }
    }
    if (prev >= 0) {
      // drain the previous tile (stage st^1) while the tensor cores run this one
      const int ps = st ^ 1;
      const bool ok = tc_wait(smem_u32(&mbar[ps]), (uint32_t)(((it - 1) >> 1) & 1));
      if (!__syncthreads_and(ok)) {
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int row = 32 * (w & 3) + lane;
      const int cb = 64 * (w >> 2);
#pragma unroll 1
      for (int half = 0; half < 2; half++) {
        const int c0 = cb + 32 * half;
        uint32_t r[32];
        const uint32_t addr = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(ps * kTcCols + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (row < n) {
          const int j = prev * kTcN + c0;
          const size_t base = (size_t)row * Jp + j;
          if (j + 32 <= J) {
#pragma unroll
            for (int q = 0; q < 8; q++) {
              float4 o = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                     __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
              float4 od = make_float4(0.f, 0.f, 0.f, 0.f);
              if (!zero) od = *(const float4 *)(Din + base + 4 * q);
              const float d0 = o.x - od.x, d1 = o.y - od.y, d2 = o.z - od.z, d3 = o.w - od.w;
              e2 = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, e2))));
              *(float4 *)(Dout + base + 4 * q) = o;
            }
          } else {
#pragma unroll
            for (int i = 0; i < 32; i++)
              if (j + i < J) {
                const float o = __uint_as_float(r[i]);
                const float d = o - (zero ? 0.f : Din[base + i]);
                e2 = fmaf(d, d, e2);
                Dout[base + i] = o;
              }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if (!have) break;
    prev = tile;
  }
  if (failed) {  // let the MMAs in flight finish before the accumulators are freed
    if (t == 0) {
      const int st = it & 1;
      tc_wait(smem_u32(&mbar[st ^ 1]), (uint32_t)(((it - 1) >> 1) & 1));  // the tile whose wait timed out
      if (blockIdx.x + it * gridDim.x < (unsigned)ntiles) tc_wait(smem_u32(&mbar[st]), (uint32_t)((it >> 1) & 1));
      atomicExch(&ds->status, OCI_E_TIMEOUT);
      ds->done = 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcCols));
  double v = (double)e2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
  __syncthreads();
  double bs = 0.0;
  if (t == 0)
    for (int i = 0; i < nthr / 32; i++) bs += red[i];
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (t == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

size_t tc_pipe_smem(const Handle &h) {
  const int n = 4 * h.N * h.G;
  const int es = h.precision == OCI_TF32_IR ? 4 : 2;
  const int parts = h.precision == OCI_TF32_IR ? 1 : 2;
  const size_t opb = (size_t)kTcM * n * es;
  const size_t need = (size_t)(h.tt.n_types + 2) * parts * opb + 1024;
  // at least 116 KB: one CTA per SM, so its 256 TMEM columns never wait for another CTA's
  const size_t floor_bytes = 116 * 1024;
  return need > floor_bytes ? need : floor_bytes;
}

bool tc_pipe_ok(const Handle &h) {
  const char *e = hook_env("OCI_TC_PIPE");  // 0: the one-tile-per-CTA kernel
  if (e && e[0] == '0') return false;
  return tc_pipe_smem(h) <= 220 * 1024;
}

static int tc_pipe_grid(const Handle &h) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = (h.J + kTcN - 1) / kTcN;
  return ntiles < sms ? ntiles : sms;
}

void launch_tc_pipe(Handle &h, cudaGraphConditionalHandle cond, int use_cond) {
  const size_t smem = tc_pipe_smem(h);
  const int grid = tc_pipe_grid(h);
  if (h.precision == OCI_TF32_IR)
    k_tc_pipe<1><<<grid, kTcPipeThreads, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.tt.n_types, h.type, h.tc_img, h.mu32,
                                                            h.z32, h.delta[0], h.delta[1], h.ds, h.partials,
                                                            h.counter, h.e_hist, cond, use_cond);
  else
    k_tc_pipe<2><<<grid, kTcPipeThreads, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.tt.n_types, h.type, h.tc_img, h.mu32,
                                                            h.z32, h.delta[0], h.delta[1], h.ds, h.partials,
                                                            h.counter, h.e_hist, cond, use_cond);
}

int tc_prepare(Handle &h) {
  if (tc_big_used(h)) return tc_big_prepare(h);
  const size_t smem = tc_smem(h);
  cudaError_t e = cudaFuncSetAttribute(k_tc_inner<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_inner<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_tc_inner)");
  if (tc_pipe_ok(h)) {
    const int ps = (int)tc_pipe_smem(h);
    e = cudaFuncSetAttribute(k_tc_pipe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_pipe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, ps);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_tc_pipe)");
  }
  return OCI_OK;
}

// Host: round FP32 to TF32 / BF16 (round to nearest even) from the bit pattern.
static float host_tf32(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  b += 0xFFFu + ((b >> 13) & 1u);
  b &= ~0x1FFFu;
  float y;
  memcpy(&y, &b, 4);
  return y;
}
static uint16_t host_bf16_bits(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}
static float bf16_bits_to_float(uint16_t h) {
  uint32_t b = (uint32_t)h << 16;
  float y;
  memcpy(&y, &b, 4);
  return y;
}

// Ainv: [T][n][n] row-major FP64 inverses of the per-type cell matrices.
int tc_build_images(Handle &h, const std::vector<double> &Ainv) {
  if (tc_big_used(h)) return tc_big_build_images(h, Ainv, host_tf32, host_bf16_bits, bf16_bits_to_float);
  const int n = 4 * h.N * h.G, T = h.tt.n_types;
  const bool tf = h.precision == OCI_TF32_IR;
  const int es = tf ? 4 : 2, parts = tf ? 1 : 2;
  const int kbytes = n * es;
  const size_t opb = (size_t)kTcM * kbytes;
  h.tc_img_bytes = parts * opb;
  std::vector<unsigned char> img((size_t)T * h.tc_img_bytes, 0);
  for (int t = 0; t < T; t++) {
    unsigned char *base = img.data() + (size_t)t * h.tc_img_bytes;
    for (int r = 0; r < n; r++)
      for (int k = 0; k < n; k++) {
        const float v = (float)Ainv[((size_t)t * n + r) * n + k];
        const uint32_t off = kmajor_off(r, k, es, kbytes);
        if (tf) {
          const float q = host_tf32(v);
          memcpy(base + off, &q, 4);
        } else {
          const uint16_t hi = host_bf16_bits(v);
          const uint16_t lo = host_bf16_bits(v - bf16_bits_to_float(hi));
          memcpy(base + off, &hi, 2);
          memcpy(base + opb + off, &lo, 2);
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
