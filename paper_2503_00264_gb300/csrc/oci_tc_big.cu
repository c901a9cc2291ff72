// oci_tc_big.cu -- tcgen05 block apply of the TF32 / BF16x3 mixed forms for cells
// with more than 128 unknowns (128 < 4NG <= 512, e.g. S16 with 8 groups).
//
// The inner sweep of the mixed forms is delta^{i+1} = A~^{-1} (r + B delta^i) per
// cell (spec: where cells share material, width and dt, the inverse of
// the cell matrix of Eqs. Aj, scatter, fullOCIlhs is applied to all of their
// right-hand sides as one dense GEMM).  For a tile of 128 cells of one type this
// is D[n x 128] = A^{-1}[n x n] . RHS[n x 128], n = 4NG.  With n up to 512 the
// inverse (1 MB in TF32) no longer fits in shared memory, so:
//   - the rows of A^{-1} are split into MT = n/128 M-tiles, each with its own
//     128-column FP32 accumulator in tensor memory (MT * 128 columns);
//   - the K dimension is walked in chunks of 32: per chunk one 1D bulk copy per
//     M-tile brings that chunk of A^{-1} (16 KB, stored chunk by chunk in the
//     K-major no-swizzle canonical layout) from global memory / L2 into shared
//     memory, while all threads build the same 32 rows of the RHS (r + B delta
//     of the 128 cells, FP32 -> TF32 or BF16 hi/lo) next to it;
//   - two stages: the MMAs of chunk k (issued by one thread, completion on an
//     mbarrier) run while the copies and the RHS of chunk k+1 are prepared;
//   - after the last chunk of a tile the CTA drains the accumulators
//     (tcgen05.ld), forms delta and the FP32 norm partial, and writes delta.
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

constexpr int kBigM = 128;      // MMA M (rows of one M-tile)
constexpr int kBigN = 128;      // MMA N (cells per tile)
constexpr int kBigKC = 32;      // K elements per chunk
constexpr int kBigBlk = 16384;  // bytes of one chunk block: 128 rows x 32 K (TF32, or BF16 hi + lo)
constexpr int kBigThreads = 256;
constexpr long long kBigSpin = 1 << 22;

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

// Byte offset of (row, k) inside one chunk block of [128 rows x 32 K]: 8-row x
// 16-byte core matrices, adjacent along K 128 B apart (LBO), 8-row groups
// (32 * es / 16) * 128 B apart (SBO).
__host__ __device__ inline uint32_t big_off(int row, int k, int es) {
  const int kc4 = 16 / es;
  return (uint32_t)((row >> 3) * (kBigKC * es / 16) * 128 + (k / kc4) * 128 + (row & 7) * 16 + (k % kc4) * es);
}

template <int KIND>  // 1 = TF32, 2 = BF16 x3
__global__ void __launch_bounds__(kBigThreads, 1) k_tc_big(
    int J, int Jp, int N, int G, int MT, int NK, const int32_t *__restrict__ type,
    const unsigned char *__restrict__ Aimg, const float *__restrict__ mu, const float *__restrict__ r32, float *D0,
    float *D1, DevState *ds, double *__restrict__ partials, unsigned *counter, double *e_hist,
    cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(1024) unsigned char smb_[];
  __shared__ __align__(8) uint64_t tma_bar[2], mma_bar[2];
  __shared__ uint32_t tslot;
  __shared__ double red[kBigThreads / 32];
  __shared__ bool s_last;
  __shared__ int s_fail;
  constexpr int es = KIND == 1 ? 4 : 2;
  constexpr int part = kBigBlk / 2;  // BF16: the lo image follows the hi image
  const int n = 4 * N * G;
  unsigned char *sm = (unsigned char *)(((uintptr_t)smb_ + 1023) & ~(uintptr_t)1023);
  const size_t stage_bytes = (size_t)(MT + 1) * kBigBlk;  // MT A blocks, then the RHS block
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (ds->done) return;  // uniform
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  const uint32_t cols = MT <= 2 ? (uint32_t)(MT * kBigN) : 512u;
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    for (int s = 0; s < 2; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&tma_bar[s])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mma_bar[s])), "r"(1));
    }
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
  const uint32_t idesc =
      (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kBigN >> 3) << 17) | ((uint32_t)(kBigM >> 4) << 24);
  const uint32_t lbo = 128, sbo = (uint32_t)(kBigKC * es / 16) * 128;
  constexpr int ksteps = kBigKC * es / 32;  // MMAs per chunk and pass (K = 8 TF32 / 16 BF16)
  constexpr int npass = KIND == 1 ? 1 : 3;  // BF16 x3: hi.hi + hi.lo + lo.hi
  // per-stage counts kept by thread 0 (copies issued, MMA groups committed)
  int n_tma[2] = {0, 0}, n_mma[2] = {0, 0};
  float e2 = 0.f;
  bool failed = false;
  int gk = 0;  // chunks started by this CTA (stage = gk & 1)
  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int j0 = tile * kBigN;
    const int tau = type[j0];
    for (int kc = 0; kc < NK; kc++, gk++) {
      const int s = gk & 1;
      unsigned char *stA = sm + (size_t)s * stage_bytes;
      unsigned char *stB = stA + (size_t)MT * kBigBlk;
      // (1) the stage is free once the MMAs of chunk gk - 2 have completed
      bool ok = true;
      if (gk >= 2) ok = big_wait(su32(&mma_bar[s]), (uint32_t)(((gk >> 1) - 1) & 1));
      if (!__syncthreads_and(ok && s_fail == 0)) {
        failed = true;
        break;
      }
      // (2) this chunk of A^{-1} for every M-tile
      if (t == 0) {
        const uint32_t bar = su32(&tma_bar[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(MT * kBigBlk)
                     : "memory");
        for (int mt = 0; mt < MT; mt++) {
          const unsigned char *src = Aimg + (((size_t)tau * MT + mt) * NK + kc) * kBigBlk;
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  su32(stA + (size_t)mt * kBigBlk)),
              "l"(reinterpret_cast<uint64_t>(src)), "r"(kBigBlk), "r"(bar)
              : "memory");
        }
        n_tma[s]++;
      }
      // (3) rows k0 .. k0+15 of the RHS of cell c = t % 128 (r + B delta, FP32), all loads first
      {
        const int c = t & (kBigN - 1), hh = t >> 7;
        const int j = j0 + c;
        const bool act = j < J;
        const int kb = kc * kBigKC + hh * 16;  // first global row
        float v[16], u[8];
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = (act && kb + i < n) ? r32[(size_t)(kb + i) * Jp + j] : 0.f;
#pragma unroll
        for (int q = 0; q < 8; q++) {  // one inflow value per (p even, p odd) row pair
          const int k = kb + 2 * q;
          const int m = (k >> 2) % N;
          u[q] = 0.f;
          if (act && !zero && k < n) {
            if (m >= N2) {
              if (j > 0) u[q] = Din[(size_t)(k + 1) * Jp + j - 1];
            } else if (j < J - 1) {
              u[q] = Din[(size_t)k * Jp + j + 1];
            }
          }
        }
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int k = kb + 2 * q;
          const int m = (k >> 2) % N;
          const float mf = mu[m < N ? m : 0];
          if (m >= N2) v[2 * q] = fmaf(mf, u[q], v[2 * q]);  // p even: mu * (R corner of cell j-1)
          else v[2 * q + 1] = fmaf(-mf, u[q], v[2 * q + 1]);  // p odd: |mu| * (L corner of cell j+1)
        }
        const int kl = hh * 16;  // row inside the chunk
        if (KIND == 1) {
#pragma unroll
          for (int g4 = 0; g4 < 16; g4 += 4)
            *(float4 *)(stB + big_off(c, kl + g4, 4)) = make_float4(v[g4], v[g4 + 1], v[g4 + 2], v[g4 + 3]);
        } else {
#pragma unroll
          for (int g8 = 0; g8 < 16; g8 += 8) {
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
            const uint32_t off = big_off(c, kl + g8, 2);
            *(uint4 *)(stB + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *(uint4 *)(stB + part + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
      }
      // (4) the RHS is visible to the tensor cores; the previous tile's drain is done
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      // (5) one thread: wait for the copies, issue the MMAs of every M-tile, commit
      if (t == 0) {
        if (!big_wait(su32(&tma_bar[s]), (uint32_t)((gk >> 1) & 1))) {
          s_fail = 1;
        } else {
          const uint32_t bA = su32(stA), bB = su32(stB);
          for (int mt = 0; mt < MT; mt++) {
            const uint32_t d_tmem = tmem + (uint32_t)(mt * kBigN);
            for (int pass = 0; pass < npass; pass++) {
              const uint32_t a0 = bA + (uint32_t)(mt * kBigBlk) + (pass == 2 ? part : 0);
              const uint32_t b0 = bB + (pass == 1 ? part : 0);
              for (int kk = 0; kk < ksteps; kk++) {
                const uint64_t ad = big_desc(a0 + kk * 256, lbo, sbo);
                const uint64_t bd = big_desc(b0 + kk * 256, lbo, sbo);
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
        }
      }
    }
    if (failed) break;
    // drain the tile: wait for its last MMA group (a commit covers all earlier MMAs)
    {
      const int sl = (gk - 1) & 1;
      __syncthreads();  // s_fail of the last chunk is visible
      bool ok = s_fail == 0 && big_wait(su32(&mma_bar[sl]), (uint32_t)(((gk - 1) >> 1) & 1));
      if (!__syncthreads_and(ok)) {
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int q4 = w & 3;             // TMEM lane quarter of this warp
      const int cb = 64 * (w >> 2);     // its 64 columns (cells)
      for (int mt = 0; mt < MT; mt++) {
        const int row = mt * kBigM + 32 * q4 + lane;
#pragma unroll 1
        for (int half = 0; half < 2; half++) {
          const int c0 = cb + 32 * half;
          uint32_t r[32];
          const uint32_t addr = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(mt * kBigN + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
              : "r"(addr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          if (row < n) {
            const int j = j0 + c0;
            const size_t base = (size_t)row * Jp + j;
            if (j + 32 <= J) {
#pragma unroll
              for (int q = 0; q < 8; q++) {
                const float4 o = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
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
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
  }
  if (failed && t == 0) {
    // let the copies and MMAs still in flight finish (bounded) before tensor memory is freed
    for (int s = 0; s < 2; s++) {
      if (n_tma[s] > 0) big_wait(su32(&tma_bar[s]), (uint32_t)((n_tma[s] - 1) & 1));
      if (n_mma[s] > 0) big_wait(su32(&mma_bar[s]), (uint32_t)((n_mma[s] - 1) & 1));
    }
    atomicExch(&ds->status, OCI_E_TIMEOUT);
    ds->done = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
  double v = (double)e2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
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

static int tc_big_mt(const Handle &h) { return (4 * h.N * h.G + kBigM - 1) / kBigM; }
static int tc_big_nk(const Handle &h) { return (4 * h.N * h.G + kBigKC - 1) / kBigKC; }

size_t tc_big_smem(const Handle &h) {
  const size_t need = 2 * (size_t)(tc_big_mt(h) + 1) * kBigBlk + 1024;
  const size_t floor_bytes = 116 * 1024;  // one CTA per SM: its tensor memory never waits for another CTA's
  return need > floor_bytes ? need : floor_bytes;
}

bool tc_big_used(const Handle &h) { return 4 * h.N * h.G > kBigM; }

int tc_big_prepare(const Handle &h) {
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
  const int grid = tc_big_grid(h), MT = tc_big_mt(h), NK = tc_big_nk(h);
  if (h.precision == OCI_TF32_IR)
    k_tc_big<1><<<grid, kBigThreads, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, MT, NK, h.type, h.tc_img, h.mu32, h.z32,
                                                        h.delta[0], h.delta[1], h.ds, h.partials, h.counter,
                                                        h.e_hist, cond, use_cond);
  else
    k_tc_big<2><<<grid, kBigThreads, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, MT, NK, h.type, h.tc_img, h.mu32, h.z32,
                                                        h.delta[0], h.delta[1], h.ds, h.partials, h.counter,
                                                        h.e_hist, cond, use_cond);
}

// Host: the per-type inverses in the chunk-major layout the kernel streams:
// block ((type * MT + mt) * NK + kc) holds rows 128 mt .. 128 mt + 127 and
// columns 32 kc .. 32 kc + 31 of A^{-1} (zero beyond n), TF32 -- or BF16 hi,
// then BF16 lo -- in the canonical K-major layout of big_off.  `round_tf32`,
// `bf16_bits` and `bf16_value` are the host roundings of the small form.
int tc_big_build_images(Handle &h, const std::vector<double> &Ainv, float (*round_tf32)(float),
                        uint16_t (*bf16_bits)(float), float (*bf16_value)(uint16_t)) {
  const int n = 4 * h.N * h.G, T = h.tt.n_types, MT = tc_big_mt(h), NK = tc_big_nk(h);
  const bool tf = h.precision == OCI_TF32_IR;
  const int es = tf ? 4 : 2;
  h.tc_img_bytes = (size_t)MT * NK * kBigBlk;
  std::vector<unsigned char> img((size_t)T * h.tc_img_bytes, 0);
  for (int t = 0; t < T; t++)
    for (int mt = 0; mt < MT; mt++)
      for (int kc = 0; kc < NK; kc++) {
        unsigned char *blk = img.data() + (((size_t)t * MT + mt) * NK + kc) * kBigBlk;
        for (int rl = 0; rl < kBigM; rl++)
          for (int kl = 0; kl < kBigKC; kl++) {
            const int r = mt * kBigM + rl, k = kc * kBigKC + kl;
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
              memcpy(blk + kBigBlk / 2 + off, &lo, 2);
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
