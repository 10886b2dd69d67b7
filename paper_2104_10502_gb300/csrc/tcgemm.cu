// Split-precision real GEMM on the 5th-generation tensor cores (tcgen05,
// kind::tf32) and the operand packing of the complex products of the
// nonlocal term (Sec. 3.3 of the paper: pseudopotential contribution to the
// Hamiltonian) for the mixed-precision path.  See tcgemm.cuh.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.h"
#include "plan.h"
#include "tc_ptx.cuh"
#include "tcgemm.cuh"

namespace qe {

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major,
// N = TC_BN, M = TC_BM.
__host__ __device__ constexpr uint32_t tf32_idesc() {
  return (1u << 4)                       // D format F32
         | (2u << 7)                     // A format TF32
         | (2u << 10)                    // B format TF32
         | ((uint32_t)(TC_BN >> 3) << 17)
         | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

// ---- the GEMM kernel ------------------------------------------------------------
// grid (Np/128, Mp/128, nsplit), block 128 (warp 0 lane 0: TMA producer; warp 1
// lane 0: MMA issuer; all four warps: epilogue).  CTA z handles K blocks
// [z*kb_per_split, min(nkb_total, (z+1)*kb_per_split)) and writes its partial
// tile to C + z*split_stride (row-major, leading dimension ldc).
__global__ void __launch_bounds__(128, 1)
k_tc_gemm_tf32x3(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                 const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                 int nkb_total, int kb_per_split, float* __restrict__ C, int ldc,
                 long long split_stride, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* tiles =
      reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(tiles + TC_STAGES * TC_STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* accb = empty + TC_STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accb + 1);
  __shared__ int s_err;
  __shared__ int s_issued;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // N tiles vary fastest across consecutive CTAs, so the CTAs that share an A
  // tile run together and read it from L2 rather than from DRAM again
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
  const int kb0 = blockIdx.z * kb_per_split;
  const int nkb = min(kb_per_split, nkb_total - kb0);
  const uint64_t limit = 2000000000ull;   // 2 s per wait

  if (threadIdx.x == 0) {
    s_err = 0;
    s_issued = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (nkb > 0 && warp == 0 && lane == 0) {
    // producer: fill the stages with TMA loads
    for (int i = 0; i < nkb; ++i) {
      const int s = i % TC_STAGES;
      const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
      if (i >= TC_STAGES && !mbar_wait(&empty[s], ph ^ 1u, limit)) {
        atomicExch(&s_err, TC_TIMEOUT_EMPTY);
        break;
      }
      if (*(volatile int*)&s_err) break;
      mbar_expect_tx(&full[s], TC_STAGE_BYTES);
      unsigned char* stg = tiles + s * TC_STAGE_BYTES;
      const int kx = (kb0 + i) * TC_BK;
      tma_load_2d(stg, &mAhi, &full[s], kx, m0);
      tma_load_2d(stg + TC_TILE_BYTES, &mAlo, &full[s], kx, m0);
      tma_load_2d(stg + 2 * TC_TILE_BYTES, &mBhi, &full[s], kx, n0);
      tma_load_2d(stg + 3 * TC_TILE_BYTES, &mBlo, &full[s], kx, n0);
      s_issued = i + 1;
    }
  } else if (nkb > 0 && warp == 1 && lane == 0) {
    // MMA issuer: three split products per K step of 8
    // descriptors: constant fields once, the start address (16-byte units) per MMA
    const uint32_t idesc = tf32_idesc();
    const uint64_t dhi = sw128_desc(0);
    const uint32_t lo0 = (smem_u32(tiles) & 0x3FFFF) >> 4;
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % TC_STAGES;
      const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, limit)) {
        atomicExch(&s_err, TC_TIMEOUT_FULL);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = lo0 + (uint32_t)s * (TC_STAGE_BYTES >> 4);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        const uint32_t off = kk * 2;
        const uint64_t ahi = dhi | (uint64_t)(sa + off);
        const uint64_t alo = dhi | (uint64_t)(sa + (TC_TILE_BYTES >> 4) + off);
        const uint64_t bhi = dhi | (uint64_t)(sa + 2 * (TC_TILE_BYTES >> 4) + off);
        const uint64_t blo = dhi | (uint64_t)(sa + 3 * (TC_TILE_BYTES >> 4) + off);
        mma_tf32(tmem, ahi, bhi, idesc, (i | kk) != 0 ? 1u : 0u);
        mma_tf32(tmem, ahi, blo, idesc, 1u);
        mma_tf32(tmem, alo, bhi, idesc, 1u);
      }
      mma_commit(&empty[s]);
    }
    if (ok) mma_commit(accb);
  }
  __syncwarp();
  // epilogue: each warp drains its 32 TMEM lanes (= 32 rows of the tile)
  bool have = false;
  if (nkb > 0) have = mbar_wait(accb, 0, limit) && *(volatile int*)&s_err == 0;
  if (nkb > 0 && !have && threadIdx.x == 0) atomicCAS(&s_err, 0, TC_TIMEOUT_ACC);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  float* crow = C + (size_t)blockIdx.z * split_stride + (size_t)(m0 + warp * 32 + lane) * ldc + n0;
  if (have) {
    for (int c = 0; c < TC_BN; c += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
      float4* dst = reinterpret_cast<float4*>(crow + c);
      dst[0] = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
      dst[1] = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]), __uint_as_float(r[7]));
      dst[2] = make_float4(__uint_as_float(r[8]), __uint_as_float(r[9]), __uint_as_float(r[10]), __uint_as_float(r[11]));
      dst[3] = make_float4(__uint_as_float(r[12]), __uint_as_float(r[13]), __uint_as_float(r[14]), __uint_as_float(r[15]));
    }
  } else if (nkb <= 0) {
    for (int c = 0; c < TC_BN; c += 4)
      *reinterpret_cast<float4*>(crow + c) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_err != 0 && threadIdx.x == 0) {
    // drain: wait (bounded) for the copies this CTA issued before releasing smem
    const int issued = s_issued;
    for (int i = max(0, issued - TC_STAGES); i < issued; ++i)
      mbar_wait(&full[i % TC_STAGES], (uint32_t)(i / TC_STAGES) & 1u, limit);
    atomicMax(status, s_err);
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN)
                 : "memory");
}

// ---- host side ----------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

int tc_get_encode(PFN_cuTensorMapEncodeTiled_v12000* fn) {
  std::call_once(g_encode_once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  if (!g_encode) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return QE_ECUDA;
  }
  if (fn) *fn = g_encode;
  return QE_OK;
}

static int get_encode() { return tc_get_encode(nullptr); }

// rows x kp FP32 matrix, K-major, box 128 rows x 32 columns, 128-byte swizzle.
static int make_map(CUtensorMap* m, const float* ptr, int rows, int kp) {
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return QE_ECUDA;
  }
  return QE_OK;
}

int tc_gemm_tf32x3(const float* Ahi, const float* Alo, const float* Bhi, const float* Blo, int Mp,
                   int Np, int Kp, int nsplit, float* C, int* status, cudaStream_t st, Prof* pf) {
  if (Mp % TC_BM || Np % TC_BN || Kp % TC_BK || Mp <= 0 || Np <= 0 || Kp <= 0 || nsplit < 1) {
    set_error("tc_gemm: bad padded sizes %d %d %d", Mp, Np, Kp);
    return QE_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(Ahi) | reinterpret_cast<uintptr_t>(Alo) |
       reinterpret_cast<uintptr_t>(Bhi) | reinterpret_cast<uintptr_t>(Blo)) & 15) {
    set_error("tc_gemm: operands must be 16-byte aligned");
    return QE_EINVAL;
  }
  int rc = get_encode();
  if (rc) return rc;
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  if ((rc = make_map(&mAhi, Ahi, Mp, Kp)) || (rc = make_map(&mAlo, Alo, Mp, Kp)) ||
      (rc = make_map(&mBhi, Bhi, Np, Kp)) || (rc = make_map(&mBlo, Blo, Np, Kp)))
    return rc;
  const int nkb = Kp / TC_BK;
  nsplit = std::min(nsplit, nkb);
  const int per = (nkb + nsplit - 1) / nsplit;
  nsplit = (nkb + per - 1) / per;   // every split non-empty
  set_max_dynamic_smem(k_tc_gemm_tf32x3);
  ProfScope ps(pf, "k_tc_gemm_tf32x3", st);
  dim3 g(Np / TC_BN, Mp / TC_BM, nsplit);
  k_tc_gemm_tf32x3<<<g, 128, TC_SMEM_BYTES, st>>>(mAhi, mAlo, mBhi, mBlo, nkb, per, C, Np,
                                                  (long long)Mp * Np, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("k_tc_gemm_tf32x3: %s", cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

int tc_gemm_splits(int Mp, int Np, int Kp) {
  const int tiles = (Mp / TC_BM) * (Np / TC_BN);
  const int nkb = Kp / TC_BK;
  // one wave: a CTA per SM (the kernel's shared memory allows no second one)
  int ns = std::max(1, 152 / std::max(1, tiles));
  ns = std::min(ns, std::max(1, nkb / 4));   // at least 4 K blocks per CTA
  const int per = (nkb + ns - 1) / ns;
  return (nkb + per - 1) / per;
}


// ---- operand packing of the complex products ---------------------------------
// Complex products are evaluated as real GEMMs over the concatenated (re, im)
// K axis, with the signs placed in the packed B operand:
//   P = conj(beta) psi^T      A[i] = [Re b_i | Im b_i],  B[n] = [Re psi_n | Im psi_n],
//                             B[nb+n] = [Im psi_n | -Re psi_n]  ->  C[i][n] = Re P, C[i][nb+n] = Im P
//   HPsi += beta^T Q          A[g] = [Re b_.(g) | Im b_.(g)],  B[n] = [Re Q_.n | -Im Q_.n],
//                             B[nb+n] = [Im Q_.n | Re Q_.n]  ->  C[g][n] = Re, C[g][nb+n] = Im
// Every value x is stored as hi = tf32(x), lo = tf32(x - hi) (round to nearest).

namespace {

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split_store(float x, float* hi, float* lo, size_t i) {
  const float h = tf32_rn(x);
  hi[i] = h;
  lo[i] = tf32_rn(x - h);
}

__device__ __forceinline__ void split_store4(const float (&x)[4], float* hi, float* lo, size_t i) {
  float4 h, l;
  h.x = tf32_rn(x[0]); l.x = tf32_rn(x[0] - h.x);
  h.y = tf32_rn(x[1]); l.y = tf32_rn(x[1] - h.y);
  h.z = tf32_rn(x[2]); l.z = tf32_rn(x[2] - h.z);
  h.w = tf32_rn(x[3]); l.w = tf32_rn(x[3] - h.w);
  *reinterpret_cast<float4*>(hi + i) = h;
  *reinterpret_cast<float4*>(lo + i) = l;
}

// Inner-product operands: the K axis of a packed row is [Re | Im] with the
// imaginary half at kh = pad4(K), so that every group of four floats lies in
// one half (16-byte stores); zero beyond K in each half and beyond 2 kh.
// One thread per four complex inputs of a row (both halves written from one
// read); grid.y = packed row.

// A[r] = [Re src_r | Im src_r], r < rows; zero rows up to Mp.
__global__ void k_pack_rows(const double2* __restrict__ src, int rows, int K, int kh, int Kp,
                            float* __restrict__ hi, float* __restrict__ lo) {
  const int r = blockIdx.y;
  const int nq = kh >> 2, nz = (Kp - 2 * kh) >> 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq + nz; q += gridDim.x * blockDim.x) {
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    if (q >= nq) {   // tail beyond 2 kh
      split_store4(re, hi, lo, (size_t)r * Kp + 2 * kh + 4 * (q - nq));
      continue;
    }
    const int k = 4 * q;
    if (r < rows) {
      const double2* s = src + (size_t)r * K + k;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (k + j < K) { const double2 v = s[j]; re[j] = (float)v.x; im[j] = (float)v.y; }
    }
    split_store4(re, hi, lo, (size_t)r * Kp + k);
    split_store4(im, hi, lo, (size_t)r * Kp + kh + k);
  }
}

// B rows n < N: [Re psi_n | Im psi_n]; rows N + n: [Im psi_n | -Re psi_n]; zero rows
// 2N .. Np.  grid.y = N + (Np - 2N): y < N writes the row pair of band y, the
// rest the zero rows.
__global__ void k_pack_psi(const double2* __restrict__ psi, int N, int K, int kh, int Kp,
                           float* __restrict__ hi, float* __restrict__ lo) {
  const int y = blockIdx.y;
  const int nq = kh >> 2, nz = (Kp - 2 * kh) >> 2;
  const size_t r0 = y < N ? (size_t)y * Kp : (size_t)(N + y) * Kp;   // zero rows: 2N + (y - N)
  const size_t r1 = (size_t)(N + y) * Kp;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq + nz; q += gridDim.x * blockDim.x) {
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    if (q >= nq || y >= N) {
      const int k = q >= nq ? 2 * kh + 4 * (q - nq) : 4 * q;
      split_store4(re, hi, lo, r0 + k);
      if (q < nq) split_store4(re, hi, lo, r0 + kh + k);
      if (y < N) split_store4(re, hi, lo, r1 + k);
      continue;
    }
    const int k = 4 * q;
    const double2* s = psi + (size_t)y * K + k;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (k + j < K) { const double2 v = s[j]; re[j] = (float)v.x; im[j] = (float)v.y; }
    split_store4(re, hi, lo, r0 + k);
    split_store4(im, hi, lo, r0 + kh + k);
    split_store4(im, hi, lo, r1 + k);
    float nre[4] = {-re[0], -re[1], -re[2], -re[3]};
    split_store4(nre, hi, lo, r1 + kh + k);
  }
}

// Transposed beta: A[g][k], k < 2 np: [Re b_k(g) | Im b_k(g)]; tiles through shared memory.
__global__ void k_pack_beta_t(const double2* __restrict__ beta, int np, int npw, int Mp, int Kp,
                              float* __restrict__ hi, float* __restrict__ lo) {
  __shared__ double2 tile[32][33];
  const int g0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  // load beta[i0 .. i0+31][g0 .. g0+31] (coalesced along g)
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, g = g0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < np && g < npw) ? beta[(size_t)i * npw + g] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  // write rows g (coalesced along k): re part at k = i, im part at k = np + i
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int g = g0 + r, i = i0 + threadIdx.x;
    if (g >= Mp || i >= np) continue;
    const double2 v = tile[threadIdx.x][r];
    split_store((float)v.x, hi, lo, (size_t)g * Kp + i);
    split_store((float)v.y, hi, lo, (size_t)g * Kp + np + i);
  }
}

// Transposed complex operand as real rows (outer products with a real right-hand
// matrix): A'[2m][k] = Re A[k][m], A'[2m+1][k] = Im A[k][m], A [K][M]; tiles
// through shared memory.
__global__ void k_pack_t_reim(const double2* __restrict__ A, int K, int M, int Kp,
                              float* __restrict__ hi, float* __restrict__ lo) {
  __shared__ double2 tile[32][33];
  const int m0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, m = m0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && m < M) ? A[(size_t)k * M + m] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int m = m0 + r, k = k0 + threadIdx.x;
    if (m >= M || k >= K) continue;
    const double2 v = tile[threadIdx.x][r];
    split_store((float)v.x, hi, lo, (size_t)(2 * m) * Kp + k);
    split_store((float)v.y, hi, lo, (size_t)(2 * m + 1) * Kp + k);
  }
}

// B rows n < N: Re Q[k][n] over k < K (Q [K][N] real-valued); zero elsewhere
__global__ void k_pack_q_real(const double2* __restrict__ Q, int K, int N, int Np, int Kp,
                              float* __restrict__ hi, float* __restrict__ lo) {
  const size_t total = (size_t)Np * Kp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / Kp), k = (int)(t % Kp);
    split_store(r < N && k < K ? (float)Q[(size_t)k * N + r].x : 0.f, hi, lo, t);
  }
}

// zero the padding of a transposed-operand matrix: rows >= rows, and columns
// k >= kvalid of the first rows
__global__ void k_pack_pad(int Mp, int Kp, int rows, int kvalid, float* __restrict__ hi,
                           float* __restrict__ lo) {
  const size_t tail = (size_t)(Mp - rows) * Kp;
  const int kc = Kp - kvalid;
  const size_t total = tail + (size_t)rows * kc;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t < tail ? (size_t)rows * Kp + t
                              : (size_t)((t - tail) / kc) * Kp + kvalid + (t - tail) % kc;
    hi[i] = 0.f;
    lo[i] = 0.f;
  }
}

// B rows n < nb: [Re Q_.n | -Im Q_.n]; rows nb + n: [Im Q_.n | Re Q_.n]; Q is [np][nb].
__global__ void k_pack_q(const double2* __restrict__ Q, int np, int nb, int Np, int Kp,
                         float* __restrict__ hi, float* __restrict__ lo) {
  const size_t total = (size_t)Np * Kp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / Kp), k = (int)(t % Kp);
    float x = 0.f;
    if (r < 2 * nb && k < 2 * np) {
      const int n = r < nb ? r : r - nb;
      const double2 q = Q[(size_t)(k < np ? k : k - np) * nb + n];
      if (r < nb) x = (float)(k < np ? q.x : -q.y);
      else x = (float)(k < np ? q.y : q.x);
    }
    split_store(x, hi, lo, t);
  }
}

// P[i][n] = (sum_s C[s][i][n], sum_s C[s][i][nb + n]) in FP64
__global__ void k_combine_p(const float* __restrict__ C, int ns, int Mp, int Np, int np, int nb,
                            double2* __restrict__ P) {
  const size_t total = (size_t)np * nb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / nb), n = (int)(t % nb);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < ns; ++s) {
      const float* c = C + (size_t)s * Mp * Np + (size_t)i * Np;
      re += (double)c[n];
      im += (double)c[nb + n];
    }
    P[t] = make_double2(re, im);
  }
}

// hpsi[n][g] += (sum_s C[s][g][n], sum_s C[s][g][nb + n]): 32 x 32 tiles of (g, n)
// through shared memory, so that both the C reads (along n) and the hpsi
// updates (along g) are coalesced.  block (32, 8), grid (ceil(npw/32), ceil(nb/32)).
__global__ void k_combine_h(const float* __restrict__ C, int ns, int Mp, int Np, int npw, int nb,
                            double2* __restrict__ hpsi) {
  __shared__ double tre[32][33], tim[32][33];
  const int g0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int g = g0 + r, n = n0 + tx;
    double re = 0.0, im = 0.0;
    if (g < npw && n < nb) {
      for (int s = 0; s < ns; ++s) {
        const float* c = C + (size_t)s * Mp * Np + (size_t)g * Np;
        re += (double)c[n];
        im += (double)c[nb + n];
      }
    }
    tre[r][tx] = re;
    tim[r][tx] = im;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int n = n0 + r, g = g0 + tx;
    if (n >= nb || g >= npw) continue;
    double2* p = hpsi + (size_t)n * npw + g;
    double2 h = *p;
    h.x += tre[tx][r];
    h.y += tim[tx][r];
    *p = h;
  }
}

// C[m][n] = (sum_s C32[s][m][n], sum_s C32[s][m][N + n]) into ld ldc (inner products)
__global__ void k_combine_inner(const float* __restrict__ C32, int ns, int Mp, int Np, int M, int N,
                                double2* __restrict__ C, int ldc) {
  const size_t total = (size_t)M * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(t / N), n = (int)(t % N);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < ns; ++s) {
      const float* c = C32 + (size_t)s * Mp * Np + (size_t)m * Np;
      re += (double)c[n];
      im += (double)c[N + n];
    }
    C[(size_t)m * ldc + n] = make_double2(re, im);
  }
}

// C[m][n] = (sum_s C32[s][m][n], 0): the real-output inner products
__global__ void k_combine_inner_real(const float* __restrict__ C32, int ns, int Mp, int Np, int M,
                                     int N, double2* __restrict__ C, int ldc) {
  const size_t total = (size_t)M * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(t / N), n = (int)(t % N);
    double re = 0.0;
    for (int s = 0; s < ns; ++s) re += (double)C32[(size_t)s * Mp * Np + (size_t)m * Np + n];
    C[(size_t)m * ldc + n] = make_double2(re, 0.0);
  }
}

// C[n][m] (+)= (-) (sum_s C32[s][m][n], sum_s C32[s][m][N + n]) (outer products)
__global__ void k_combine_outer(const float* __restrict__ C32, int ns, int Mp, int Np, int M, int N,
                                double2* __restrict__ C, int ldc, int alpha_neg, int beta) {
  const size_t total = (size_t)N * M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(t / M), m = (int)(t % M);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < ns; ++s) {
      const float* c = C32 + (size_t)s * Mp * Np + (size_t)m * Np;
      re += (double)c[n];
      im += (double)c[N + n];
    }
    if (alpha_neg) { re = -re; im = -im; }
    double2* p = C + (size_t)n * ldc + m;
    if (beta) { const double2 o = *p; re += o.x; im += o.y; }
    *p = make_double2(re, im);
  }
}

// C[n][m] (+)= (-) (sum_s C32[s][2m][n], sum_s C32[s][2m+1][n]) (outer products
// with a real right-hand matrix)
__global__ void k_combine_outer_reim(const float* __restrict__ C32, int ns, int Mp, int Np, int M,
                                     int N, double2* __restrict__ C, int ldc, int alpha_neg,
                                     int beta) {
  const size_t total = (size_t)N * M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(t / M), m = (int)(t % M);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < ns; ++s) {
      const float* c = C32 + (size_t)s * Mp * Np + (size_t)(2 * m) * Np + n;
      re += (double)c[0];
      im += (double)c[Np];
    }
    if (alpha_neg) { re = -re; im = -im; }
    double2* p = C + (size_t)n * ldc + m;
    if (beta) { const double2 o = *p; re += o.x; im += o.y; }
    *p = make_double2(re, im);
  }
}

int grid_of(size_t total) {
  return (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, 152 * 16));
}

}  // namespace

static inline int pad_to(int x, int m) { return (x + m - 1) / m * m; }
// K layout of the inner-product operands: imaginary half at kh = pad4(K), rows of
// Kp = pad(2 kh) floats
static inline int kh_of(int K) { return pad_to(K, 4); }
static inline int kcat(int K) { return pad_to(2 * kh_of(K), TC_BK); }
static inline dim3 pack_grid(int Kp, int kh, int rows) {
  const int items = (kh + (Kp - 2 * kh)) / 4;
  return dim3((unsigned)std::max(1, std::min((items + 255) / 256, 64)), (unsigned)rows);
}

// Packed beta operands (both GEMMs); they depend only on beta, np and npw, so a
// caller that applies the same operator repeatedly packs them once.
size_t nonlocal_tc_beta_bytes(int np, int npw) {
  const size_t Mp = pad_to(np, TC_BM), Kp = kcat(npw);
  const size_t Mp2 = pad_to(npw, TC_BM), Kp2 = pad_to(2 * np, TC_BK);
  return 2 * Mp * Kp * 4 + 2 * Mp2 * Kp2 * 4 + 4 * 256;
}

size_t nonlocal_tc_bytes(int np, int nb, int npw) {
  const size_t Mp = pad_to(np, TC_BM), Kp = kcat(npw), Np = pad_to(2 * nb, TC_BN);
  const size_t Mp2 = pad_to(npw, TC_BM), Kp2 = pad_to(2 * np, TC_BK);
  const size_t ns1 = tc_gemm_splits((int)Mp, (int)Np, (int)Kp), ns2 = tc_gemm_splits((int)Mp2, (int)Np, (int)Kp2);
  size_t b = 0;
  b += 2 * Np * Kp * 4 + ns1 * Mp * Np * 4;                          // inner product
  b += 2 * Np * Kp2 * 4 + ns2 * Mp2 * Np * 4;                        // outer product
  b += 2 * (size_t)np * nb * 16 + 64 * 256;                          // P, Q, alignment
  return b;
}

// Nonlocal term on the tensor cores: hpsi += beta^T D (conj(beta) psi^T).
// bpack (nonlocal_tc_beta_bytes) holds the packed beta operands; they are
// (re)written when pack_beta is true.
int nonlocal_tc(const double* beta, const double* dmat, const double* psi, double* hpsi, int np,
                int nb, int npw, void* bpack, bool pack_beta, void* work, size_t work_bytes,
                int* status, cudaStream_t st, Prof* pf, bool real_p) {
  if (np <= 0 || nb <= 0) return QE_OK;
  if (nonlocal_tc_bytes(np, nb, npw) > work_bytes) {
    set_error("nonlocal_tc: workspace too small");
    return QE_EINVAL;
  }
  const int Mp = pad_to(np, TC_BM), Kp = kcat(npw), Np = pad_to(2 * nb, TC_BN), kh = kh_of(npw);
  const int Mp2 = pad_to(npw, TC_BM), Kp2 = pad_to(2 * np, TC_BK);
  const int ns1 = tc_gemm_splits(Mp, Np, Kp), ns2 = tc_gemm_splits(Mp2, Np, Kp2);
  char* p = static_cast<char*>(bpack);
  auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~(size_t)255; return q; };
  float* ahi = (float*)take((size_t)Mp * Kp * 4);
  float* alo = (float*)take((size_t)Mp * Kp * 4);
  float* a2hi = (float*)take((size_t)Mp2 * Kp2 * 4);
  float* a2lo = (float*)take((size_t)Mp2 * Kp2 * 4);
  p = static_cast<char*>(work);
  float* bhi = (float*)take((size_t)Np * Kp * 4);
  float* blo = (float*)take((size_t)Np * Kp * 4);
  float* c1 = (float*)take((size_t)ns1 * Mp * Np * 4);
  float* b2hi = (float*)take((size_t)Np * Kp2 * 4);
  float* b2lo = (float*)take((size_t)Np * Kp2 * 4);
  float* c2 = (float*)take((size_t)ns2 * Mp2 * Np * 4);
  double2* P = (double2*)take((size_t)np * nb * 16);
  double2* Q = (double2*)take((size_t)np * nb * 16);
  if (pack_beta) {
    ProfScope ps(pf, "k_pack_beta", st);
    k_pack_rows<<<pack_grid(Kp, kh, Mp), 256, 0, st>>>((const double2*)beta, np, npw, kh, Kp, ahi, alo);
    k_pack_pad<<<grid_of((size_t)(Mp2 - npw) * Kp2 + (size_t)npw * (Kp2 - 2 * np)), 256, 0, st>>>(
        Mp2, Kp2, npw, 2 * np, a2hi, a2lo);
    dim3 gt((Mp2 + 31) / 32, (np + 31) / 32);
    k_pack_beta_t<<<gt, dim3(32, 8), 0, st>>>((const double2*)beta, np, npw, Mp2, Kp2, a2hi, a2lo);
    if (pf) pf->launches += 2;
  }
  {
    ProfScope ps(pf, "k_pack_psi", st);
    k_pack_psi<<<pack_grid(Kp, kh, Np - nb), 256, 0, st>>>((const double2*)psi, nb, npw, kh, Kp, bhi, blo);
  }
  int rc = tc_gemm_tf32x3(ahi, alo, bhi, blo, Mp, Np, Kp, ns1, c1, status, st, pf);
  if (rc) return rc;
  {
    ProfScope ps(pf, "k_combine_p", st);
    k_combine_p<<<grid_of((size_t)np * nb), 256, 0, st>>>(c1, ns1, Mp, Np, np, nb, P);
  }
  rc = dmul(dmat, (const double*)P, (double*)Q, np, nb, st, pf, real_p);
  if (rc) return rc;
  {
    ProfScope ps(pf, "k_pack_q", st);
    k_pack_q<<<grid_of((size_t)Np * Kp2), 256, 0, st>>>(Q, np, nb, Np, Kp2, b2hi, b2lo);
  }
  rc = tc_gemm_tf32x3(a2hi, a2lo, b2hi, b2lo, Mp2, Np, Kp2, ns2, c2, status, st, pf);
  if (rc) return rc;
  {
    ProfScope ps(pf, "k_combine_h", st);
    k_combine_h<<<dim3((npw + 31) / 32, (nb + 31) / 32), dim3(32, 8), 0, st>>>(c2, ns2, Mp2, Np, npw,
                                                                             nb, (double2*)hpsi);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("nonlocal_tc: %s", cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

// ---- general complex products (mixed path subspace products) -------------------------
// inner: C[m][n] = sum_k conj(A[m][k]) B[n][k], rows of A and B contiguous in k
// (leading dimension K); outer: C[n][m] (+)= (-) sum_k A[k][m] B[k][n] with A
// [K][M] and B [K][N] dense.  FP32-accurate (TF32 x3) on the tensor cores.
size_t tc_inner_bytes(int M, int N, int K) {
  if (M <= 0 || N <= 0) return 0;
  const size_t Mp = pad_to(M, TC_BM), Kp = kcat(K), Np = pad_to(2 * N, TC_BN);
  const size_t ns = tc_gemm_splits((int)Mp, (int)Np, (int)Kp);
  return 2 * Mp * Kp * 4 + 2 * Np * Kp * 4 + ns * Mp * Np * 4 + 8 * 256;
}

size_t tc_outer_bytes(int M, int N, int K) {
  if (M <= 0 || N <= 0) return 0;
  const size_t Mp = pad_to(M, TC_BM), Kp = pad_to(2 * K, TC_BK), Np = pad_to(2 * N, TC_BN);
  const size_t ns = tc_gemm_splits((int)Mp, (int)Np, (int)Kp);
  return 2 * Mp * Kp * 4 + 2 * Np * Kp * 4 + ns * Mp * Np * 4 + 8 * 256;
}

int tc_inner(const double* A, const double* B, int M, int N, int K, double* C, int ldc, void* work,
             size_t work_bytes, int* status, cudaStream_t st, Prof* pf, bool real_out) {
  if (M <= 0 || N <= 0) return QE_OK;
  if (tc_inner_bytes(M, N, K) > work_bytes) {
    set_error("tc_inner: workspace too small");
    return QE_EINVAL;
  }
  // real output: Re(a^+ b) is the real dot product of the [Re | Im] rows, so B
  // needs only its [Re | Im] rows (half the GEMM's columns)
  const int Mp = pad_to(M, TC_BM), Kp = kcat(K), Np = pad_to(real_out ? N : 2 * N, TC_BN);
  const int kh = kh_of(K);
  const int ns = tc_gemm_splits(Mp, Np, Kp);
  char* p = static_cast<char*>(work);
  auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~(size_t)255; return q; };
  float* ahi = (float*)take((size_t)Mp * Kp * 4);
  float* alo = (float*)take((size_t)Mp * Kp * 4);
  float* bhi = (float*)take((size_t)Np * Kp * 4);
  float* blo = (float*)take((size_t)Np * Kp * 4);
  float* c = (float*)take((size_t)ns * Mp * Np * 4);
  {
    ProfScope ps(pf, "k_tc_pack", st);
    k_pack_rows<<<pack_grid(Kp, kh, Mp), 256, 0, st>>>((const double2*)A, M, K, kh, Kp, ahi, alo);
    if (real_out)
      k_pack_rows<<<pack_grid(Kp, kh, Np), 256, 0, st>>>((const double2*)B, N, K, kh, Kp, bhi, blo);
    else
      k_pack_psi<<<pack_grid(Kp, kh, Np - N), 256, 0, st>>>((const double2*)B, N, K, kh, Kp, bhi, blo);
    if (pf) pf->launches += 1;
  }
  int rc = tc_gemm_tf32x3(ahi, alo, bhi, blo, Mp, Np, Kp, ns, c, status, st, pf);
  if (rc) return rc;
  ProfScope ps(pf, "k_tc_combine", st);
  if (real_out)
    k_combine_inner_real<<<grid_of((size_t)M * N), 256, 0, st>>>(c, ns, Mp, Np, M, N, (double2*)C, ldc);
  else
    k_combine_inner<<<grid_of((size_t)M * N), 256, 0, st>>>(c, ns, Mp, Np, M, N, (double2*)C, ldc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error("tc_inner: %s", cudaGetErrorString(e)); return QE_ECUDA; }
  return QE_OK;
}

size_t tc_outer_real_bytes(int M, int N, int K) {
  if (M <= 0 || N <= 0) return 0;
  const size_t Mp = pad_to(2 * M, TC_BM), Kp = pad_to(K, TC_BK), Np = pad_to(N, TC_BN);
  const size_t ns = tc_gemm_splits((int)Mp, (int)Np, (int)Kp);
  return 2 * Mp * Kp * 4 + 2 * Np * Kp * 4 + ns * Mp * Np * 4 + 8 * 256;
}

// The outer product with a real right-hand matrix B: the real and imaginary parts
// of A's columns are separate GEMM rows over a real K axis, 2M x N x K instead of
// M x 2N x 2K (half the tensor-core work).
int tc_outer_real(const double* A, const double* B, int M, int N, int K, double* C, int ldc,
                  int alpha_neg, int beta, void* work, size_t work_bytes, int* status,
                  cudaStream_t st, Prof* pf) {
  if (M <= 0 || N <= 0) return QE_OK;
  if (tc_outer_real_bytes(M, N, K) > work_bytes) {
    set_error("tc_outer_real: workspace too small");
    return QE_EINVAL;
  }
  const int Mp = pad_to(2 * M, TC_BM), Kp = pad_to(K, TC_BK), Np = pad_to(N, TC_BN);
  const int ns = tc_gemm_splits(Mp, Np, Kp);
  char* p = static_cast<char*>(work);
  auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~(size_t)255; return q; };
  float* ahi = (float*)take((size_t)Mp * Kp * 4);
  float* alo = (float*)take((size_t)Mp * Kp * 4);
  float* bhi = (float*)take((size_t)Np * Kp * 4);
  float* blo = (float*)take((size_t)Np * Kp * 4);
  float* c = (float*)take((size_t)ns * Mp * Np * 4);
  {
    ProfScope ps(pf, "k_tc_pack", st);
    k_pack_pad<<<grid_of((size_t)(Mp - 2 * M) * Kp + (size_t)2 * M * (Kp - K)), 256, 0, st>>>(
        Mp, Kp, 2 * M, K, ahi, alo);
    dim3 gt((M + 31) / 32, (K + 31) / 32);
    k_pack_t_reim<<<gt, dim3(32, 8), 0, st>>>((const double2*)A, K, M, Kp, ahi, alo);
    k_pack_q_real<<<grid_of((size_t)Np * Kp), 256, 0, st>>>((const double2*)B, K, N, Np, Kp, bhi, blo);
    if (pf) pf->launches += 2;
  }
  int rc = tc_gemm_tf32x3(ahi, alo, bhi, blo, Mp, Np, Kp, ns, c, status, st, pf);
  if (rc) return rc;
  ProfScope ps(pf, "k_tc_combine", st);
  k_combine_outer_reim<<<grid_of((size_t)M * N), 256, 0, st>>>(c, ns, Mp, Np, M, N, (double2*)C,
                                                             ldc, alpha_neg, beta);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error("tc_outer_real: %s", cudaGetErrorString(e)); return QE_ECUDA; }
  return QE_OK;
}

int tc_outer(const double* A, const double* B, int M, int N, int K, double* C, int ldc,
             int alpha_neg, int beta, void* work, size_t work_bytes, int* status, cudaStream_t st,
             Prof* pf) {
  if (M <= 0 || N <= 0) return QE_OK;
  if (tc_outer_bytes(M, N, K) > work_bytes) {
    set_error("tc_outer: workspace too small");
    return QE_EINVAL;
  }
  const int Mp = pad_to(M, TC_BM), Kp = pad_to(2 * K, TC_BK), Np = pad_to(2 * N, TC_BN);
  const int ns = tc_gemm_splits(Mp, Np, Kp);
  char* p = static_cast<char*>(work);
  auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~(size_t)255; return q; };
  float* ahi = (float*)take((size_t)Mp * Kp * 4);
  float* alo = (float*)take((size_t)Mp * Kp * 4);
  float* bhi = (float*)take((size_t)Np * Kp * 4);
  float* blo = (float*)take((size_t)Np * Kp * 4);
  float* c = (float*)take((size_t)ns * Mp * Np * 4);
  {
    ProfScope ps(pf, "k_tc_pack", st);
    k_pack_pad<<<grid_of((size_t)(Mp - M) * Kp + (size_t)M * (Kp - 2 * K)), 256, 0, st>>>(
        Mp, Kp, M, 2 * K, ahi, alo);
    dim3 gt((Mp + 31) / 32, (K + 31) / 32);
    k_pack_beta_t<<<gt, dim3(32, 8), 0, st>>>((const double2*)A, K, M, Mp, Kp, ahi, alo);
    k_pack_q<<<grid_of((size_t)Np * Kp), 256, 0, st>>>((const double2*)B, K, N, Np, Kp, bhi, blo);
    if (pf) pf->launches += 2;
  }
  int rc = tc_gemm_tf32x3(ahi, alo, bhi, blo, Mp, Np, Kp, ns, c, status, st, pf);
  if (rc) return rc;
  ProfScope ps(pf, "k_tc_combine", st);
  k_combine_outer<<<grid_of((size_t)M * N), 256, 0, st>>>(c, ns, Mp, Np, M, N, (double2*)C, ldc,
                                                        alpha_neg, beta);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error("tc_outer: %s", cudaGetErrorString(e)); return QE_ECUDA; }
  return QE_OK;
}

}  // namespace qe
