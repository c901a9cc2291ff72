// oci_mixed.cu -- mixed-precision form of the OCI step: inner sweeps on an FP32
// correction, FP64 refinement.
//
// With A = L_c - S block diagonal and B the lagged-inflow coupling (Eq. oci),
// plain OCI is Psi^{l+1} = A^{-1}(c + B Psi^l).  From an outer iterate Psi with
// FP64 residual r = c + B Psi - A Psi, the iterates of plain OCI are
// Psi^{l+i} = Psi + delta^i with
//     delta^0 = 0,   delta^{i+1} = A^{-1}(r + B delta^i),
// and the per-sweep change e_i = ||delta^{i+1} - delta^i||_2 equals plain OCI's
// ||Psi^{l+i+1} - Psi^{l+i}||_2.  The inner recursion runs in FP32 (structured
// cell solve with FP32 tables); every few sweeps the correction is folded into
// the FP64 iterate and the residual is recomputed in FP64, which removes the
// FP32 error accumulated so far (defect correction).  The stop rule of Sec. 2.1
// is applied to every inner sweep, so sweep counts track the FP64 form.
//
// A refinement happens after k_max inner sweeps, or once e < theta * (first e
// of the block) -- by then the FP32 correction has gained about -log10(theta)
// digits and more inner sweeps would only resolve FP32 rounding -- and at
// convergence.  The stop rule is accepted only on a sweep whose correction is
// small (first sweep after a refinement, or a block that began below tol), so
// the committed iterate carries no more than low-precision rounding of a tiny
// correction; this costs at most one extra sweep per step.  FP64 is kept for Psi,
// the residual, the norm accumulation, the balance tallies and the carry.
#include <cuda.h>
#include <math.h>

#include "oci_device.cuh"

namespace oci {

// ---------------------------------------------------------------- inner sweep
// delta_out = A~^{-1}(r + B delta_in) through the structured solve in FP32:
// t = z + Cin u, y = sum_m w t, s = Mp y, delta = t + Linv s, where z = A~-block
// solve of r precomputed by the outer kernel (z = Linv r).  The correction has
// zero incident flux at the slab ends (the boundary values live in r).
__global__ void __launch_bounds__(256) k_mx_inner(int J, int Jp, int N, int G, int P,
                                                  const int32_t *__restrict__ type, const float *__restrict__ Linv,
                                                  const float *__restrict__ Cin, const float *__restrict__ Mp,
                                                  const float *__restrict__ w, const float *__restrict__ z, float *D0,
                                                  float *D1, DevState *ds, double *__restrict__ partials,
                                                  unsigned *counter, double *e_hist,
                                                  cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ float smf[];
  __shared__ double red[32];
  __shared__ bool s_last;
  const int CB = blockDim.x;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P;
  const int NP = N / P, m0 = ch * NP;
  const int j = blockIdx.x * CB + cl;
  if (ds->done) return;
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const float *__restrict__ Din = dcur ? D1 : D0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  float *t_s = smf;
  float *y_s = smf + (size_t)G * N * 4 * CB;
  const bool active = j < J;
  const int tau = active ? type[j] : 0;
  const int N2 = N / 2;
  const size_t tb = (size_t)tau * G * N;
  float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
  if (active) {
#pragma unroll 4
    for (int m = m0; m < m0 + NP; m++) {
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      float uk = 0.f, uh = 0.f;
      if (!zero) {
        if (m >= N2) {
          if (j > 0) {
            uk = Din[base + (size_t)Jp - 1];
            uh = Din[base + 3 * (size_t)Jp - 1];
          }
        } else if (j < J - 1) {
          uk = Din[base + 1];
          uh = Din[base + 2 * (size_t)Jp + 1];
        }
      }
      const float *C = Cin + (tb + gm) * 8;
      const float t0 = fmaf(C[1], uh, fmaf(C[0], uk, z[base]));
      const float t1 = fmaf(C[3], uh, fmaf(C[2], uk, z[base + (size_t)Jp]));
      const float t2 = fmaf(C[5], uh, fmaf(C[4], uk, z[base + 2 * (size_t)Jp]));
      const float t3 = fmaf(C[7], uh, fmaf(C[6], uk, z[base + 3 * (size_t)Jp]));
      float *ts = t_s + (size_t)(gm * 4) * CB + cl;
      ts[0] = t0;
      ts[CB] = t1;
      ts[2 * CB] = t2;
      ts[3 * CB] = t3;
      const float wm = w[m];
      y0 = fmaf(wm, t0, y0);
      y1 = fmaf(wm, t1, y1);
      y2 = fmaf(wm, t2, y2);
      y3 = fmaf(wm, t3, y3);
    }
    float *ys = y_s + (size_t)(gy * 4) * CB + cl;
    ys[0] = y0;
    ys[CB] = y1;
    ys[2 * CB] = y2;
    ys[3 * CB] = y3;
  }
  __syncthreads();
  float e2 = 0.f;
  if (active) {
    const int G4 = 4 * G;
    const float *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4) * G4;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int k = 0; k < G4; k++) {
      const int gp = k >> 2, q = k & 3;
      float yk = y_s[(size_t)((gp * P) * 4 + q) * CB + cl];
      for (int c = 1; c < P; c++) yk += y_s[(size_t)((gp * P + c) * 4 + q) * CB + cl];
      s0 = fmaf(M[k], yk, s0);
      s1 = fmaf(M[G4 + k], yk, s1);
      s2 = fmaf(M[2 * G4 + k], yk, s2);
      s3 = fmaf(M[3 * G4 + k], yk, s3);
    }
#pragma unroll 4
    for (int m = m0; m < m0 + NP; m++) {
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      const float *L = Linv + (tb + gm) * 16;
      const float *ts = t_s + (size_t)(gm * 4) * CB + cl;
#pragma unroll
      for (int p = 0; p < 4; p++) {
        const float o = fmaf(L[p * 4 + 3], s3, fmaf(L[p * 4 + 2], s2, fmaf(L[p * 4 + 1], s1, fmaf(L[p * 4 + 0], s0, ts[p * CB]))));
        const float d = zero ? o : o - Din[base + (size_t)p * Jp];
        e2 = fmaf(d, d, e2);
        Dout[base + (size_t)p * Jp] = o;
      }
    }
  }
  // FP64 accumulation of the per-thread FP32 partial sums
  double v = (double)e2;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double bs = 0.0;
  if (tid == 0)
    for (int i = 0; i < (nthr + 31) / 32; i++) bs += red[i];
  // the block that finishes last reduces all partials and applies the stop rule
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (tid == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

// ---------------------------------------------------------------- inner sweep, TMA-staged
// The same FP32 inner sweep with the tile's operands brought in by the tensor
// memory accelerator: per tile of kTmaCells cells, one 2D bulk tensor copy
// moves z[0:R][j0:j0+64] and one moves delta_in[0:R][j0-4:j0+68] (the halo
// columns j0-1 and j0+64 are inside; x starts on a 16-byte boundary; columns
// outside the array read as zero, which is the correction's zero inflow at the
// slab ends) into shared memory, completing on an mbarrier.  A persistent CTA
// double-buffers the stages: the copy of its next tile is in flight while the
// current one is computed.  R = 4NG <= 256 (one box per operand).
constexpr int kTmaCells = 64;
constexpr int kTmaHalo = 4;                    // columns each side of the delta box
constexpr int kTmaDW = kTmaCells + 2 * kTmaHalo;  // delta box width
constexpr long long kTmaSpin = 1 << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__global__ void __launch_bounds__(256) k_mx_inner_tma(const __grid_constant__ CUtensorMap tmZ,
                                                      const __grid_constant__ CUtensorMap tmD0,
                                                      const __grid_constant__ CUtensorMap tmD1, int J, int Jp, int N,
                                                      int G, int P, const int32_t *__restrict__ type,
                                                      const float *__restrict__ Linv, const float *__restrict__ Cin,
                                                      const float *__restrict__ Mp, const float *__restrict__ w,
                                                      float *D0, float *D1, DevState *ds,
                                                      double *__restrict__ partials, unsigned *counter,
                                                      double *e_hist, cudaGraphConditionalHandle cond,
                                                      int use_cond) {
  extern __shared__ __align__(1024) unsigned char smraw_[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ double red[32];
  __shared__ bool s_last;
  // stage buffers start on a 1024-byte boundary (the launch reserves 1 KiB extra)
  unsigned char *smraw = (unsigned char *)(((uintptr_t)smraw_ + 1023) & ~(uintptr_t)1023);
  const int R = 4 * N * G;
  const int cl = threadIdx.x, gy = threadIdx.y;
  const int g = gy / P, ch = gy % P;
  const int NP = N / P, m0 = ch * NP;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  if (ds->done) return;  // uniform
  const bool zero = ds->refine || ds->blk_i == 0;
  const int dcur = ds->dcur;
  const CUtensorMap *tmDin = dcur ? &tmD1 : &tmD0;
  float *__restrict__ Dout = dcur ? D0 : D1;
  // stage layout: z [R][64] then delta [R][72], each stage 1024-aligned
  const size_t zbytes = (size_t)R * kTmaCells * 4, dbytes = (size_t)R * kTmaDW * 4;
  const size_t stage_bytes = (zbytes + dbytes + 1023) / 1024 * 1024;
  float *y_s = (float *)(smraw + 2 * stage_bytes);  // [G*P*4][64]
  const uint32_t tx = (uint32_t)(zbytes + (zero ? 0 : dbytes));
  const int ntiles = (J + kTmaCells - 1) / kTmaCells;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  auto issue = [&](int tile, int st) {
    const uint32_t bar = smem_addr(&mbar[st]);
    unsigned char *base = smraw + st * stage_bytes;
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
    tma_load_2d(smem_addr(base), &tmZ, tile * kTmaCells, 0, bar);
    if (!zero) tma_load_2d(smem_addr(base + zbytes), tmDin, tile * kTmaCells - kTmaHalo, 0, bar);
  };
  const int N2 = N / 2;
  const int G4 = 4 * G;
  float e2 = 0.f;
  int it = 0;
  bool failed = false;
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
    const int st = it & 1;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    if (tid == 0 && tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x, st ^ 1);
    uint32_t ok = 0;
    for (long long k = 0; k < kTmaSpin && !ok; k++) {
      asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                   : "=r"(ok)
                   : "r"(smem_addr(&mbar[st])), "r"(parity)
                   : "memory");
    }
    if (!__syncthreads_and(ok)) {  // the same decision in every thread
      failed = true;
      break;
    }
    const float *zs = (const float *)(smraw + st * stage_bytes);
    const float *ds_ = (const float *)(smraw + st * stage_bytes + zbytes);
    const int j = tile * kTmaCells + cl;
    const bool active = j < J;
    const int tau = active ? type[j] : 0;
    const size_t tb = (size_t)tau * G * N;
    auto dval = [&](int r, int col) -> float { return zero ? 0.f : ds_[r * kTmaDW + col]; };
    float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
    if (active) {
      for (int m = m0; m < m0 + NP; m++) {
        const int gm = g * N + m;
        float uk, uh;
        if (m >= N2) {  // upstream R corner of cell j-1 (zero beyond the slab end)
          uk = dval(gm * 4 + 1, cl + kTmaHalo - 1);
          uh = dval(gm * 4 + 3, cl + kTmaHalo - 1);
        } else {  // upstream L corner of cell j+1
          uk = (j < J - 1) ? dval(gm * 4 + 0, cl + kTmaHalo + 1) : 0.f;
          uh = (j < J - 1) ? dval(gm * 4 + 2, cl + kTmaHalo + 1) : 0.f;
        }
        const float *C = Cin + (tb + gm) * 8;
        const float wm = w[m];
        y0 = fmaf(wm, fmaf(C[1], uh, fmaf(C[0], uk, zs[(gm * 4 + 0) * kTmaCells + cl])), y0);
        y1 = fmaf(wm, fmaf(C[3], uh, fmaf(C[2], uk, zs[(gm * 4 + 1) * kTmaCells + cl])), y1);
        y2 = fmaf(wm, fmaf(C[5], uh, fmaf(C[4], uk, zs[(gm * 4 + 2) * kTmaCells + cl])), y2);
        y3 = fmaf(wm, fmaf(C[7], uh, fmaf(C[6], uk, zs[(gm * 4 + 3) * kTmaCells + cl])), y3);
      }
    }
    y_s[(gy * 4 + 0) * kTmaCells + cl] = y0;
    y_s[(gy * 4 + 1) * kTmaCells + cl] = y1;
    y_s[(gy * 4 + 2) * kTmaCells + cl] = y2;
    y_s[(gy * 4 + 3) * kTmaCells + cl] = y3;
    __syncthreads();
    if (active) {
      const float *M = Mp + (size_t)tau * G4 * G4 + (size_t)(g * 4) * G4;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      for (int k = 0; k < G4; k++) {
        const int gp = k >> 2, q = k & 3;
        float yk = 0.f;
        for (int c = 0; c < P; c++) yk += y_s[((gp * P + c) * 4 + q) * kTmaCells + cl];
        s0 = fmaf(M[k], yk, s0);
        s1 = fmaf(M[G4 + k], yk, s1);
        s2 = fmaf(M[2 * G4 + k], yk, s2);
        s3 = fmaf(M[3 * G4 + k], yk, s3);
      }
      for (int m = m0; m < m0 + NP; m++) {
        const int gm = g * N + m;
        float uk, uh;
        if (m >= N2) {
          uk = dval(gm * 4 + 1, cl + kTmaHalo - 1);
          uh = dval(gm * 4 + 3, cl + kTmaHalo - 1);
        } else {
          uk = (j < J - 1) ? dval(gm * 4 + 0, cl + kTmaHalo + 1) : 0.f;
          uh = (j < J - 1) ? dval(gm * 4 + 2, cl + kTmaHalo + 1) : 0.f;
        }
        const float *C = Cin + (tb + gm) * 8;
        const float *L = Linv + (tb + gm) * 16;
#pragma unroll
        for (int p = 0; p < 4; p++) {
          const float t = fmaf(C[p * 2 + 1], uh, fmaf(C[p * 2 + 0], uk, zs[(gm * 4 + p) * kTmaCells + cl]));
          const float o = fmaf(L[p * 4 + 3], s3, fmaf(L[p * 4 + 2], s2, fmaf(L[p * 4 + 1], s1, fmaf(L[p * 4 + 0], s0, t))));
          const float d = o - dval(gm * 4 + p, cl + kTmaHalo);
          e2 = fmaf(d, d, e2);
          Dout[(size_t)(gm * 4 + p) * Jp + j] = o;
        }
      }
    }
    __syncthreads();  // stage st and y_s are free for the next tile
  }
  if (failed && tid == 0) {
    atomicExch(&ds->status, OCI_E_TIMEOUT);
    ds->done = 1;
  }
  double v = (double)e2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double bs = 0.0;
  if (tid == 0)
    for (int i = 0; i < (nthr + 31) / 32; i++) bs += red[i];
  if (publish_partial(partials, blockIdx.x, bs, counter, gridDim.x, &s_last)) {
    const double tot = block_sum_fixed(partials, gridDim.x, red);
    if (tid == 0) {
      *counter = 0;
      finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
    }
  }
}

size_t mx_tma_smem(const Handle &h, int P) {
  const int R = 4 * h.N * h.G;
  const size_t zbytes = (size_t)R * kTmaCells * 4, dbytes = (size_t)R * kTmaDW * 4;
  const size_t stage_bytes = (zbytes + dbytes + 1023) / 1024 * 1024;
  return 2 * stage_bytes + (size_t)h.G * P * 4 * kTmaCells * 4 + 1024;
}

const void *k_mx_inner_tma_ptr() { return (const void *)k_mx_inner_tma; }

// Encode the three tensor maps (z and the two delta buffers, [R rows][Jp cols] FP32).
int mx_tma_setup(Handle &h) {
  const int R = 4 * h.N * h.G;
  if (R > 256) return OCI_OK;  // one box per operand only
  typedef CUresult (*Encode)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  Encode enc = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&enc, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !enc) return OCI_OK;  // no TMA path: keep the plain kernel
  const cuuint64_t dims[2] = {(cuuint64_t)h.Jp, (cuuint64_t)R};
  const cuuint64_t strides[1] = {(cuuint64_t)h.Jp * 4};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint32_t boxz[2] = {(cuuint32_t)kTmaCells, (cuuint32_t)R};
  const cuuint32_t boxd[2] = {(cuuint32_t)kTmaDW, (cuuint32_t)R};
  CUresult r1 = enc(&h.tm_z, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.z32, dims, strides, boxz, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = enc(&h.tm_d[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.delta[0], dims, strides, boxd, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r3 = enc(&h.tm_d[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h.delta[1], dims, strides, boxd, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS || r3 != CUDA_SUCCESS) return OCI_OK;
  e = cudaFuncSetAttribute(k_mx_inner_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_mx_inner_tma)");
  h.tma_ok = true;
  return OCI_OK;
}

// ---------------------------------------------------------------- outer (FP64)
// mode 0: residual of Psi[cur] (start of a step, correction zero)
// mode 1: if ds->refine: Psi[cur^1] = Psi[cur] + delta[dcur]; unless the step is
//         done, residual of Psi[cur^1]
// mode 2: if ds->blk_i > 0: Psi[cur^1] = Psi[cur] + delta[dcur] (apply only)
// The residual r = c + s + inflow - L_c Psi (Eqs. oci, Aj, rhs_sg, scatter) is
// formed in FP64 and z = Linv r (FP32) is stored for the inner sweeps.
__global__ void __launch_bounds__(256) k_mx_outer(int J, int Jp, int N, int G, const int32_t *__restrict__ type,
                                                  const double *__restrict__ Lco, const double *__restrict__ Kap,
                                                  const float *__restrict__ Linv32, const double *__restrict__ w,
                                                  const double *__restrict__ mu, const double *__restrict__ inc,
                                                  const double *__restrict__ cvec, double *Psi0, double *Psi1,
                                                  const float *D0, const float *D1, const DevState *__restrict__ ds,
                                                  int mode, int store_r, float *__restrict__ z32) {
  extern __shared__ double smd[];
  const int CB = blockDim.x;
  const int cl = threadIdx.x, g = threadIdx.y;
  if (mode == 1 && !ds->refine) return;  // the common case: a small grid exits at once
  if (mode == 2 && ds->blk_i == 0) return;
  const bool apply = mode != 0;
  const bool resid = mode == 0 || (mode == 1 && !ds->done);
  const int cur = ds->cur;
  const double *__restrict__ Pin = cur ? Psi1 : Psi0;
  double *__restrict__ Pout = cur ? Psi0 : Psi1;
  const float *__restrict__ Dl = ds->dcur ? D1 : D0;
  const int N2 = N / 2;
  const int ntiles = (J + CB - 1) / CB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j = tile * CB + cl;
    const bool active = j < J;
    const int tau = active ? type[j] : 0;
    double ph[4] = {0.0, 0.0, 0.0, 0.0};
    if (active) {
      for (int m = 0; m < N; m++) {
        const int gm = g * N + m;
        const size_t base = (size_t)gm * 4 * Jp + j;
        const double wm = w[m];
#pragma unroll
        for (int p = 0; p < 4; p++) {
          double v = Pin[base + (size_t)p * Jp];
          if (apply) {
            v += (double)Dl[base + (size_t)p * Jp];
            Pout[base + (size_t)p * Jp] = v;
          }
          ph[p] = fma(wm, v, ph[p]);
        }
      }
    }
    if (!resid) continue;  // uniform
    double *ph_s = smd;    // [G*4][CB]
    __syncthreads();       // previous tile's readers are done
#pragma unroll
    for (int p = 0; p < 4; p++) ph_s[(size_t)(g * 4 + p) * CB + cl] = ph[p];
    __syncthreads();
    if (!active) continue;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int gp = 0; gp < G; gp++) {
      const double k = Kap[((size_t)tau * G + gp) * G + g];
#pragma unroll
      for (int p = 0; p < 4; p++) s[p] = fma(k, ph_s[(size_t)(gp * 4 + p) * CB + cl], s[p]);
    }
    const double *__restrict__ P = apply ? Pout : Pin;
    for (int m = 0; m < N; m++) {
      const int gm = g * N + m;
      const size_t base = (size_t)gm * 4 * Jp + j;
      const double v0 = P[base], v1 = P[base + (size_t)Jp], v2 = P[base + 2 * (size_t)Jp],
                   v3 = P[base + 3 * (size_t)Jp];
      const double *L = Lco + ((size_t)tau * G * N + gm) * 5;  // a, mu/2, alpha/2, alpha, alpha+a
      const double a = L[0], hm = L[1], ha = L[2], al = L[3], aa = L[4];
      double r0 = cvec[base] + s[0];
      double r1 = cvec[base + (size_t)Jp] + s[1];
      double r2 = cvec[base + 2 * (size_t)Jp] + s[2];
      double r3 = cvec[base + 3 * (size_t)Jp] + s[3];
      if (m >= N2) {  // mu > 0: upstream R corner of cell j-1 into rows 0, 2
        double uk, uh;
        if (j > 0) {
          const size_t nb = base - 1;
          uk = Pin[nb + (size_t)Jp];
          uh = Pin[nb + 3 * (size_t)Jp];
          if (apply) {
            uk += (double)Dl[nb + (size_t)Jp];
            uh += (double)Dl[nb + 3 * (size_t)Jp];
          }
        } else {
          uk = inc[gm * 2 + 0];
          uh = inc[gm * 2 + 1];
        }
        r0 = fma(mu[m], uk, r0);
        r2 = fma(mu[m], uh, r2);
      } else {  // mu < 0: upstream L corner of cell j+1 into rows 1, 3
        double uk, uh;
        if (j < J - 1) {
          const size_t nb = base + 1;
          uk = Pin[nb];
          uh = Pin[nb + 2 * (size_t)Jp];
          if (apply) {
            uk += (double)Dl[nb];
            uh += (double)Dl[nb + 2 * (size_t)Jp];
          }
        } else {
          uk = inc[(G * N + gm) * 2 + 0];
          uh = inc[(G * N + gm) * 2 + 1];
        }
        r1 = fma(-mu[m], uk, r1);
        r3 = fma(-mu[m], uh, r3);
      }
      // r -= L_c Psi  (rows of Eq. Aj)
      r0 = fma(-a, v0, fma(-hm, v1, fma(-ha, v2, r0)));
      r1 = fma(hm, v0, fma(-a, v1, fma(-ha, v3, r1)));
      r2 = fma(al, v0, fma(-aa, v2, fma(-hm, v3, r2)));
      r3 = fma(al, v1, fma(hm, v2, fma(-aa, v3, r3)));
      const float f0 = (float)r0, f1 = (float)r1, f2 = (float)r2, f3 = (float)r3;
      if (store_r) {  // the tensor-core inner sweep applies the dense inverse to r itself
        z32[base] = f0;
        z32[base + (size_t)Jp] = f1;
        z32[base + 2 * (size_t)Jp] = f2;
        z32[base + 3 * (size_t)Jp] = f3;
        continue;
      }
      const float *Li = Linv32 + ((size_t)tau * G * N + gm) * 16;
#pragma unroll
      for (int p = 0; p < 4; p++)
        z32[base + (size_t)p * Jp] = fmaf(Li[p * 4 + 3], f3, fmaf(Li[p * 4 + 2], f2, fmaf(Li[p * 4 + 1], f1, Li[p * 4 + 0] * f0)));
    }
  }
}

// ---------------------------------------------------------------- control
__global__ void __launch_bounds__(kFinalizeThreads) k_mx_finalize(const double *__restrict__ partials, int n,
                                                                    DevState *ds, double *e_hist,
                                                                    cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double red[32];
  if (ds->done) {
    if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  const double tot = block_sum_fixed(partials, n, red);
  if (threadIdx.x == 0) finish_mixed(ds, e_hist, sqrt(tot), cond, use_cond);
}

// kind 0: settle a pending refinement (flip Psi, zero correction)
// kind 1: after an apply-only outer kernel (mode 2), flip Psi
__global__ void k_mx_settle(DevState *ds, int kind) {
  if (kind == 0) {
    if (ds->refine) {
      ds->cur ^= 1;
      ds->refine = 0;
      ds->blk_i = 0;
    }
  } else if (ds->blk_i > 0) {
    ds->cur ^= 1;
    ds->blk_i = 0;
  }
}

static void mx_shape(const Handle &h, int &cb, int &P) {
  cb = h.mx_cb;
  P = h.mx_P;
  if (cb > 0) return;
  P = 1;
  cb = 128;
  while (cb > 1 && ((size_t)cb * h.G > 256 || sweep_smem(h.N, h.G, cb, 1, 4) > 96 * 1024)) cb /= 2;
}

int tc_partials(const Handle &h);
int mx_partials(const Handle &h) {
  if (h.precision != OCI_FP32_IR) return tc_partials(h);
  if (h.mx_tma) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_inner_tma, kTmaCells * h.G * h.mx_P,
                                                  mx_tma_smem(h, h.mx_P));
    const int ntiles = (h.J + kTmaCells - 1) / kTmaCells;
    const int grid = sms * (per > 0 ? per : 1);
    return grid < ntiles ? grid : ntiles;
  }
  int cb, P;
  mx_shape(h, cb, P);
  return (h.J + cb - 1) / cb;
}

// One inner sweep including its norm reduction, stop rule and refinement
// decision (fused into the last block).
void launch_mx_inner(Handle &h, cudaGraphConditionalHandle cond, int use_cond) {
  if (h.mx_tma) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int P = h.mx_P;
    const size_t smem = mx_tma_smem(h, P);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mx_inner_tma, kTmaCells * h.G * P, smem);
    const int ntiles = (h.J + kTmaCells - 1) / kTmaCells;
    int grid = sms * (per > 0 ? per : 1);
    if (grid > ntiles) grid = ntiles;
    k_mx_inner_tma<<<grid, dim3(kTmaCells, h.G * P), smem, h.stream>>>(
        h.tm_z, h.tm_d[0], h.tm_d[1], h.J, h.Jp, h.N, h.G, P, h.type, h.tt.Linv32, h.tt.Cin32, h.tt.Mp32, h.w32,
        h.delta[0], h.delta[1], h.ds, h.partials, h.counter, h.e_hist, cond, use_cond);
    return;
  }
  int cb, P;
  mx_shape(h, cb, P);
  dim3 block(cb, h.G * P);
  k_mx_inner<<<(h.J + cb - 1) / cb, block, sweep_smem(h.N, h.G, cb, P, 4), h.stream>>>(
      h.J, h.Jp, h.N, h.G, P, h.type, h.tt.Linv32, h.tt.Cin32, h.tt.Mp32, h.w32, h.z32, h.delta[0], h.delta[1], h.ds,
      h.partials, h.counter, h.e_hist, cond, use_cond);
}

void launch_mx_outer(Handle &h, int mode) {
  int cb = 128;
  while (cb > 1 && cb * h.G > 256) cb /= 2;
  dim3 block(cb, h.G);
  const size_t smem = (size_t)cb * h.G * 4 * sizeof(double);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = (h.J + cb - 1) / cb;
  const int grid = ntiles < 4 * sms ? ntiles : 4 * sms;  // grid-stride over tiles
  k_mx_outer<<<grid, block, smem, h.stream>>>(h.J, h.Jp, h.N, h.G, h.type, h.tt.Lco, h.tt.Kap,
                                                             h.tt.Linv32, h.w, h.mu, h.inc, h.tc, h.Psi[0], h.Psi[1],
                                                             h.delta[0], h.delta[1], h.ds, mode,
                                                             h.precision != OCI_FP32_IR, h.z32);
}

void launch_mx_finalize(Handle &h, cudaGraphConditionalHandle cond, int use_cond) {
  k_mx_finalize<<<1, kFinalizeThreads, 0, h.stream>>>(h.partials, mx_partials(h), h.ds, h.e_hist, cond, use_cond);
}

void launch_mx_settle(Handle &h, int kind) { k_mx_settle<<<1, 1, 0, h.stream>>>(h.ds, kind); }

const void *k_mx_inner_ptr() { return (const void *)k_mx_inner; }

}  // namespace oci
