// FP64-accurate complex matrix products on the BF16 tensor cores (tcgen05,
// kind::f16) by exact operand splitting — the Ozaki scheme (Ozaki, Ogita,
// Oishi & Rump, Numer. Algorithms 59, 2012) — for the FP64 path's projector
// products of the nonlocal term (Sec. 3.3 of the paper: pseudopotential
// contribution to the Hamiltonian).
//
// GB300 runs FP64 at ~1.2 TFLOP/s on either the vector or the DMMA pipe, and
// BF16 at ~1.9 PFLOP/s.  Every row r of an operand is scaled by 2^-e_r (e_r the
// exponent bound of its largest entry) and written as S = 8 slices of 7 bits:
//   round(x 2^(56-e_r)) 2^-56 = sum_t q_t 2^-7(t+1),  q_t integer,
//   |q_1| <= 128, |q_t>1| <= 64 (balanced digits), each q_t exact in BF16
// (the rounding to 2^-56 of the row maximum is below the dropped terms).  A product of slices t and u is an integer below
// 2^14; the tensor cores sum such products exactly in FP32 as long as the sum
// stays below 2^24, which holds for the pairs of one "diagonal" t + u = d over
// a K chunk of 384 (at most 10 * 2^12 per K step on the longest diagonal).  The
// pairs with t + u <= S - 1 (0-based; 36 of 64) are kept: the dropped ones
// weigh below 2^-55 of |row max| * |column max| per term.  Each diagonal has its
// own FP32 accumulator in TMEM (8 x 64 columns = all 512); after every chunk the
// epilogue warps add them, scaled by 2^-7(d+2), into FP64 registers.
//
// Complex products are real GEMMs on interleaved (re, im) K axes:
//   inner  P = conj(A) B^T:  A'[m] = (ar, ai)_k,  B'[2n] = (br, bi)_k,  B'[2n+1] = (bi, -br)_k
//   outer  C = A^T B:        A'[m] = (ar, ai)_k,  B'[2n] = (br, -bi)_k, B'[2n+1] = (bi, br)_k
// so that column 2n of the real product is Re and 2n+1 is Im of complex column n.
// Where only Re P is wanted (bands real in r, k = 0): B'[n] = (br, bi)_k, so that
// columns 2p and 2p+1 are Re P of complex columns 2p and 2p+1 (half the work).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "common.h"
#include "plan.h"
#include "tc_ptx.cuh"

namespace qe {

constexpr int OZ_S = 8;                 // slices per operand
constexpr int OZ_BM = 128;              // rows of A per CTA (TMEM lanes)
constexpr int OZ_BN = 64;               // rows of B per CTA (columns of one accumulator)
constexpr int OZ_BK = 64;               // K per step: one 128-byte swizzle row of BF16
constexpr int OZ_KPC = 6;               // K steps per exact FP32 chunk (384)
constexpr int OZ_ASTAGES = 6;
constexpr int OZ_A_BYTES = OZ_BM * OZ_BK * 2;            // 16 KiB: one A slice tile
constexpr int OZ_B_BYTES = OZ_BN * OZ_BK * 2;            // 8 KiB: one B slice tile
constexpr int OZ_BSTAGE_BYTES = OZ_S * OZ_B_BYTES;       // all B slices of one K step
constexpr int OZ_SMEM_BYTES = OZ_ASTAGES * OZ_A_BYTES + 2 * OZ_BSTAGE_BYTES + 1024 + 256;
constexpr int OZ_THREADS = 320;         // warps 0-7 epilogue, 8 TMA producer, 9 MMA issuer
constexpr int OZ_ECOLS = OZ_BN / 2;     // accumulator columns per epilogue warp
enum { OZ_OK = 0, OZ_TIMEOUT = 4 };

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major,
// N = OZ_BN, M = OZ_BM.
__host__ __device__ constexpr uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
         ((uint32_t)(OZ_BM >> 4) << 24);
}
// ... with N = n columns (a multiple of 16, at most 256)
__host__ __device__ constexpr uint32_t oz_idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1.
template <int I, int N, typename F>
__device__ __forceinline__ void oz_sfor_from(F& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    oz_sfor_from<I + 1, N>(f);
  }
}
template <int N, typename F>
__device__ __forceinline__ void oz_sfor(F&& f) {
  oz_sfor_from<0, N>(f);
}

// The same with the A operand kept in the tensor core's collector buffer across
// consecutive MMAs of one A tile: C = 1 fills it (read from shared memory), 2
// uses it, 3 uses it for the last time.
template <int C>
__device__ __forceinline__ void mma_bf16_coll(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accum) {
  if constexpr (C == 1)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  else if constexpr (C == 2)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  else if constexpr (C == 3)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  else
    mma_bf16(dtmem, adesc, bdesc, idesc, accum);
}

// 2^e as a double for the exponent range of normal numbers.
__device__ __forceinline__ double pow2(int e) {
  e = max(-1022, min(1023, e));
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// A row exponent; 0x80808080 marks an all-zero column of a transposed slicing.
__device__ __forceinline__ int oz_exp(int e) { return e == (int)0x80808080 ? 0 : e; }

// ---- the GEMM kernel ----------------------------------------------------------
// C'[m][j] = sum_k A'[m][k] B'[j][k] for one 128 x 64 tile and one K range.
// A slices: rows t * Mp + m of mapA; B slices: rows t * Np + j of mapB.
// Output: complex pairs (C'[m][2n], C'[m][2n+1]) to out[z * zstride + n * ldo + m]
// for m < M, n < N (n = j / 2), negated if alpha_neg, added to the old value if
// beta; scaled by 2^(eA[m] + eB[n]) (emode 0: one exponent per column pair), or
// column j by 2^(eA[m] + eB[j]) (emode 1).  emode 2: real outputs, C'[m][j] x
// 2^(eA[m] + eB[j]) to the real (m even) or imaginary (m odd) part of
// out[z * zstride + j * ldo + m / 2], for m < M, j < N.  grid (Np / 64, Mp / 128, nsplit); CTA z takes K steps
// [z * ks_per_split, min(nks, (z + 1) * ks_per_split)).
__global__ void __launch_bounds__(OZ_THREADS, 1)
k_oz_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
          int Mp, int Np, int nks, int ks_per_split, const int* __restrict__ eA,
          const int* __restrict__ eB, double2* __restrict__ out, int ldo, long long zstride, int M,
          int N, int alpha_neg, int beta, int emode, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;                                   // OZ_ASTAGES x 16 KiB
  unsigned char* sB = base + OZ_ASTAGES * OZ_A_BYTES;          // 2 x 64 KiB
  uint64_t* afull = reinterpret_cast<uint64_t*>(sB + 2 * OZ_BSTAGE_BYTES);
  uint64_t* aempty = afull + OZ_ASTAGES;
  uint64_t* bfull = aempty + OZ_ASTAGES;
  uint64_t* bempty = bfull + 2;
  uint64_t* accfull = bempty + 2;
  uint64_t* accempty_hi = accfull + 1;   // diagonals 4 .. 7 drained
  uint64_t* accempty_lo = accfull + 2;   // diagonals 0 .. 3 drained
  uint64_t* mmadone = accfull + 3;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mmadone + 1);
  __shared__ int s_err, s_issued_a, s_issued_b;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * OZ_BN, m0 = blockIdx.y * OZ_BM;
  const int ks0 = blockIdx.z * ks_per_split;
  const int nk = max(0, min(ks_per_split, nks - ks0));
  const int nchunks = (nk + OZ_KPC - 1) / OZ_KPC;
  const uint64_t limit = 2000000000ull;   // 2 s per wait

  if (threadIdx.x == 0) {
    s_err = 0;
    s_issued_a = 0;
    s_issued_b = 0;
    for (int s = 0; s < OZ_ASTAGES; ++s) {
      mbar_init(&afull[s], 1);
      mbar_init(&aempty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bfull[s], 1);
      mbar_init(&bempty[s], 1);
    }
    mbar_init(accfull, 1);
    mbar_init(accempty_hi, 8);
    mbar_init(accempty_lo, 8);
    mbar_init(mmadone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == 8 && lane == 0 && nk > 0) {
    // producer: per K step, all B slices (one stage of the B ring), then the
    // A slices one per stage of the A ring
    int j = 0;
    for (int i = 0; i < nk && !*(volatile int*)&s_err; ++i) {
      const int sb = i & 1;
      if (i >= 2 && !mbar_wait(&bempty[sb], ((uint32_t)(i >> 1) & 1u) ^ 1u, limit)) {
        atomicExch(&s_err, OZ_TIMEOUT);
        break;
      }
      const int kx = (ks0 + i) * OZ_BK;
      mbar_expect_tx(&bfull[sb], OZ_BSTAGE_BYTES);
      for (int t = 0; t < OZ_S; ++t)
        tma_load_2d(sB + sb * OZ_BSTAGE_BYTES + t * OZ_B_BYTES, &mapB, &bfull[sb], kx, t * Np + n0);
      s_issued_b = i + 1;
      for (int t = 0; t < OZ_S; ++t, ++j) {
        const int sa = j % OZ_ASTAGES;
        if (j >= OZ_ASTAGES &&
            !mbar_wait(&aempty[sa], ((uint32_t)(j / OZ_ASTAGES) & 1u) ^ 1u, limit)) {
          atomicExch(&s_err, OZ_TIMEOUT);
          break;
        }
        mbar_expect_tx(&afull[sa], OZ_A_BYTES);
        tma_load_2d(sA + sa * OZ_A_BYTES, &mapA, &afull[sa], kx, t * Mp + m0);
        s_issued_a = j + 1;
      }
    }
  } else if (warp == 9 && lane == 0 && nk > 0) {
    // MMA issuer: for every K step and A slice t, the pairs (t, u), u <= S-1-t,
    // into the accumulator of diagonal d = t + u.  The accumulators of the
    // diagonals t .. S-1 are consecutive in TMEM (64 columns each) and the B
    // slices u = 0 .. S-1-t consecutive in shared memory (64 rows each), so one
    // MMA of N = 64 (S - t) columns -- in pieces of at most 256 -- computes all
    // pairs of slice t: 12 MMAs per 16-deep k slab instead of 36 (one thread
    // issues them, ~57 cycles each, which had bounded the 128 x 64 x 16 form at
    // 47 % of the tensor pipe).  The loops are unrolled: every descriptor offset
    // is a constant; the A ring has 6 stages (0.499 -> 0.459 ms against 4).
    const uint64_t dhi = sw128_desc(0);
    const uint32_t a_lo0 = (smem_u32(sA) & 0x3FFFF) >> 4, b_lo0 = (smem_u32(sB) & 0x3FFFF) >> 4;
    int c = 0;
    bool ok = true;
    for (int i = 0; i < nk && ok; ++i) {
      const bool cstart = (i % OZ_KPC) == 0;
      // the first K step of a chunk after the first: the epilogue drains
      // diagonals 4 .. 7 first, so this step's pairs into them go first and the
      // pairs into 0 .. 3 of slices 0 .. 3 wait for the rest of the drain
      const bool split = cstart && i > 0;
      if (split && !mbar_wait(accempty_hi, (uint32_t)(c - 1) & 1u, limit)) {
        atomicExch(&s_err, OZ_TIMEOUT);
        ok = false;
        break;
      }
      const int sb = i & 1;
      if (!mbar_wait(&bfull[sb], (uint32_t)(i >> 1) & 1u, limit)) {
        atomicExch(&s_err, OZ_TIMEOUT);
        ok = false;
        break;
      }
      const uint32_t b_lo = b_lo0 + (uint32_t)sb * (OZ_BSTAGE_BYTES >> 4);
      const int jbase = i * OZ_S;   // A slices consumed before this K step
      oz_sfor<OZ_S>([&](auto T) {
        constexpr int t = decltype(T)::value;
        if (!ok) return;
        const int j = jbase + t, sa = j % OZ_ASTAGES;
        if (!mbar_wait(&afull[sa], (uint32_t)(j / OZ_ASTAGES) & 1u, limit)) {
          atomicExch(&s_err, OZ_TIMEOUT);
          ok = false;
          return;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_lo = a_lo0 + (uint32_t)sa * (OZ_A_BYTES >> 4);
        if constexpr (t < 4) {
          if (split) {
            // pairs of slice t into diagonals 4 .. 7: B slices 4-t .. 7-t, N = 256
#pragma unroll
            for (int kk = 0; kk < OZ_BK / 16; ++kk) {
              const uint64_t ad = dhi | (uint64_t)(a_lo + kk * 2);
              const uint64_t bd = dhi | (uint64_t)(b_lo + (4 - t) * (OZ_B_BYTES >> 4) + kk * 2);
              mma_bf16(tmem + (uint32_t)(4 * OZ_BN), ad, bd, oz_idesc_n(4 * OZ_BN),
                       (t == 0 && kk == 0) ? 0u : 1u);
            }
            if constexpr (t == 3) {
              if (!mbar_wait(accempty_lo, (uint32_t)(c - 1) & 1u, limit)) {
                atomicExch(&s_err, OZ_TIMEOUT);
                ok = false;
                return;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              // pairs of slices 0 .. 3 into diagonals t2 .. 3: B slices 0 .. 3-t2
              oz_sfor<4>([&](auto T2) {
                constexpr int t2 = decltype(T2)::value;
                const int sa2 = (jbase + t2) % OZ_ASTAGES;
                const uint32_t a_lo2 = a_lo0 + (uint32_t)sa2 * (OZ_A_BYTES >> 4);
#pragma unroll
                for (int kk = 0; kk < OZ_BK / 16; ++kk) {
                  const uint64_t ad = dhi | (uint64_t)(a_lo2 + kk * 2);
                  const uint64_t bd = dhi | (uint64_t)(b_lo + kk * 2);
                  mma_bf16(tmem + (uint32_t)(t2 * OZ_BN), ad, bd, oz_idesc_n((4 - t2) * OZ_BN),
                           (t2 == 0 && kk == 0) ? 0u : 1u);
                }
                mma_commit(&aempty[sa2]);
              });
            }
            return;
          }
        }
#pragma unroll
        for (int kk = 0; kk < OZ_BK / 16; ++kk) {
          const uint64_t ad = dhi | (uint64_t)(a_lo + kk * 2);
          const uint32_t acc = (cstart && t == 0 && kk == 0) ? 0u : 1u;
          constexpr int npiece = (OZ_S - t + 3) / 4;
          oz_sfor<npiece>([&](auto Pc) {
            constexpr int pc = decltype(Pc)::value, u0 = 4 * pc;
            constexpr int nu = (OZ_S - t - u0) < 4 ? (OZ_S - t - u0) : 4;
            constexpr uint32_t idn = oz_idesc_n(nu * OZ_BN);
            // two pieces on one A slab: it enters the collector buffer once
            constexpr int coll = npiece == 1 ? 0 : (pc == 0 ? 1 : 3);
            const uint32_t dt = tmem + (uint32_t)((t + u0) * OZ_BN);
            const uint64_t bd = dhi | (uint64_t)(b_lo + u0 * (OZ_B_BYTES >> 4) + kk * 2);
            mma_bf16_coll<coll>(dt, ad, bd, idn, acc);
          });
        }
        mma_commit(&aempty[sa]);
      });
      if (!ok) break;
      mma_commit(&bempty[sb]);
      if ((i % OZ_KPC) == OZ_KPC - 1 || i == nk - 1) {
        mma_commit(accfull);
        ++c;
      }
    }
    // every MMA issued so far has completed once this barrier flips
    mma_commit(mmadone);
    mbar_wait(mmadone, 0, limit);
  }
  __syncwarp();

  if (warp < 8) {
    // epilogue warp: TMEM lanes of quarter (warp % 4), columns [c0, c0 + 32)
    const int quarter = warp & 3, c0 = (warp >> 2) * OZ_ECOLS;
    // Integer accumulation in units of 2^-unit of the scaled product (no FP64
    // instruction per chunk: GB300's FP64 pipe would bound the drain).  A
    // chunk's exact diagonal sums combine, four at a time, into
    //   T0 = ((S_0 128 + S_1) 128 + S_2) 128 + S_3   (units 2^-35),
    //   T1 = ((S_4 128 + S_5) 128 + S_6) 128 + S_7   (units 2^-63),
    // added as T0 2^(unit-35) + round(T1 2^(unit-63)).  The CTA's whole value
    // is below its K range K_cta (|a|, |b| < 1 after scaling), so unit =
    // min(52, 62 - bits(K_cta)) keeps the sum below 2^62; the rounding adds at
    // most 2^-(unit+1) per chunk of 384 terms, below 2^-53 per term of the K
    // sum when unit >= 45 (K_cta < 2^17), the order of the dropped slice pairs.
    const int kbits = 64 - __clzll((long long)nk * OZ_BK);
    const int unit = max(36, min(52, 62 - kbits));
    const int sh0 = unit - 35, sh1 = 63 - unit;
    const long long half1 = 1ll << (sh1 - 1);
    long long acc[OZ_ECOLS];
#pragma unroll
    for (int q = 0; q < OZ_ECOLS; ++q) acc[q] = 0;
    bool ok = true;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
    for (int c = 0; c < nchunks; ++c) {
      if (!mbar_wait(accfull, (uint32_t)c & 1u, limit) || *(volatile int*)&s_err) {
        if (lane == 0) atomicCAS(&s_err, 0, OZ_TIMEOUT);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // diagonals 4 .. 7 first (T1), then 0 .. 3 (T0): the MMAs of the next
      // chunk into 4 .. 7 start while 0 .. 3 are read (integer sums: exact in
      // any order)
#pragma unroll
      for (int gi = 0; gi < 2; ++gi) {
        const int g = 1 - gi;
#pragma unroll
        for (int cb = 0; cb < OZ_ECOLS / 8; ++cb) {
          uint32_t r[4][8];
#pragma unroll
          for (int dd = 0; dd < 4; ++dd)
            tmem_ld8_nowait(lane_base + (uint32_t)((4 * g + dd) * OZ_BN + cb * 8), r[dd]);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            long long T = __float2int_rn(__uint_as_float(r[0][q]));
#pragma unroll
            for (int dd = 1; dd < 4; ++dd) T = T * 128 + __float2int_rn(__uint_as_float(r[dd][q]));
            acc[cb * 8 + q] += g ? ((T + half1) >> sh1) : (T << sh0);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(g ? accempty_hi : accempty_lo);
      }
    }
    const int m = m0 + quarter * 32 + lane;
    if (ok && m < M && emode == 2) {
      // real outputs: GEMM row m is the real (m even) or imaginary (m odd) part
      // of complex output row m / 2, GEMM column j a real column
      const int ea = oz_exp(eA[m]);
      double* o = reinterpret_cast<double*>(out + (size_t)blockIdx.z * zstride) + (m & 1);
#pragma unroll
      for (int c = 0; c < OZ_ECOLS; ++c) {
        const int j = n0 + c0 + c;
        if (j >= N) break;
        double v = __ll2double_rn(acc[c]) * pow2(ea + oz_exp(eB[j]) - unit);
        if (alpha_neg) v = -v;
        double* p = o + 2 * ((size_t)j * ldo + (m >> 1));
        if (beta) v += *p;
        *p = v;
      }
    } else if (ok && m < M) {
      const int ecol = emode;
      const int ea = oz_exp(eA[m]);
      double2* o = out + (size_t)blockIdx.z * zstride + m;
#pragma unroll
      for (int q = 0; q < OZ_ECOLS / 2; ++q) {
        const int n = ((n0 + c0) >> 1) + q;
        if (n >= N) break;
        const int eb0 = oz_exp(eB[ecol ? 2 * n : n]);
        const int eb1 = ecol ? oz_exp(eB[2 * n + 1]) : eb0;
        double2 v = make_double2(__ll2double_rn(acc[2 * q]) * pow2(ea + eb0 - unit),
                                 __ll2double_rn(acc[2 * q + 1]) * pow2(ea + eb1 - unit));
        if (alpha_neg) { v.x = -v.x; v.y = -v.y; }
        double2* p = o + (size_t)n * ldo;
        if (beta) { const double2 old = *p; v.x += old.x; v.y += old.y; }
        *p = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_err != 0 && threadIdx.x == 0) {
    // drain: wait (bounded) for the copies this CTA issued before releasing smem
    const int ia = s_issued_a, ib = s_issued_b;
    for (int j = max(0, ia - OZ_ASTAGES); j < ia; ++j)
      mbar_wait(&afull[j % OZ_ASTAGES], (uint32_t)(j / OZ_ASTAGES) & 1u, limit);
    for (int i = max(0, ib - 2); i < ib; ++i) mbar_wait(&bfull[i & 1], (uint32_t)(i >> 1) & 1u, limit);
    atomicMax(status, s_err);
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
}

// ---- slicing ------------------------------------------------------------------
// All integer: GB300's FP64 pipe (which also runs FP64 min/max and conversions)
// would otherwise bound the slicing instead of memory.

// |x| as an ordered integer key (the IEEE magnitude bits).
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Exponent bound from magnitude bits: the smallest e with |x| < 2^e (0 for 0).
__device__ __forceinline__ int exp_bound_bits(unsigned long long b) {
  if (b == 0) return 0;
  const int E = (int)(b >> 52);
  if (E > 0) return E - 1022;                  // 2^(E-1023) <= |x| < 2^(E-1022)
  return -1074 + (64 - __clzll((long long)b));   // subnormal
}

__device__ __forceinline__ int exp_bound(double mx) { return exp_bound_bits(mag_bits(mx)); }

// BF16 bits of an integer v, |v| <= 128: its float has at most 8 significant
// bits, so the upper half of the float's bits is exactly the BF16 value.
__device__ __forceinline__ unsigned short bf16_of_int(int v) {
  return (unsigned short)(__float_as_uint(__int2float_rn(v)) >> 16);
}

// The S slices of x 2^-e: F = round(|x| 2^(56-e)) < 2^56 in balanced base-128
// digits, least significant first (digits in [-64, 63], the leading one in
// [0, 128]), with the sign of x; q[t] are BF16 bit patterns.  F is handled as
// two 28-bit halves (four digits each) in 32-bit arithmetic.
__device__ __forceinline__ void slices_of(double x, int e, unsigned short* q) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  int Ee = E;
  if (E > 0) m |= 1ull << 52;
  else Ee = 1;
  // |x| = m 2^(Ee-1075);  F = m 2^(Ee-1075+56-e) rounded
  const int s = 1019 - Ee + e;
  unsigned long long F;
  if (s <= 0) F = m << (-s);
  else if (s >= 64) F = 0;
  else F = (m + (1ull << (s - 1))) >> s;
  const int sg = (b >> 63) ? -1 : 1;
  unsigned lo = (unsigned)(F & 0xFFFFFFFull), hi = (unsigned)(F >> 28);
  int carry = 0;
#pragma unroll
  for (int t = OZ_S - 1; t >= 1; --t) {
    unsigned& w = t >= 4 ? lo : hi;
    int v = (int)(w & 127u) + carry;
    w >>= 7;
    carry = v >= 64 ? 1 : 0;
    v -= carry << 7;
    q[t] = bf16_of_int(sg * v);
  }
  q[0] = bf16_of_int(sg * ((int)hi + carry));
}

__device__ __forceinline__ unsigned pack2(unsigned short lo, unsigned short hi) {
  return (unsigned)lo | ((unsigned)hi << 16);
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, t, o);
      t = w > t ? w : t;
    }
    if (threadIdx.x == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// Row slicing: input row r of a complex [rows][K] matrix (leading dimension ld,
// complex units).  form 0: output row r = (x, y)_k; form 1: rows 2r = (x, y)_k
// and 2r+1 = (y, -x)_k.  Q is [S][rows_out_p][Kp] BF16 (K padding zeroed), e[r]
// the row's exponent.  One CTA per input row (padding rows included: zeros).
constexpr int OZ_ROW_CHUNK = 2048;   // complex elements of a row per CTA

// Row exponents of a complex [rows][K] matrix: grid (rows, ceil(K / 2048)); the
// CTAs of a row merge their exponent bounds with atomicMax (monotonic in the
// maximum) into e[r], which holds 0x80808080 beforehand (kept by all-zero rows).
__global__ void __launch_bounds__(256) k_oz_rowmax(const double2* __restrict__ src, int ld, int K,
                                                   int* __restrict__ e) {
  __shared__ unsigned long long sh[33];
  const int r = blockIdx.x;
  const double2* row = src + (size_t)r * ld;
  const int k0 = blockIdx.y * OZ_ROW_CHUNK, k1 = min(K, k0 + OZ_ROW_CHUNK);
  unsigned long long mx = 0;
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double2 v = row[k];
    const unsigned long long a = mag_bits(v.x), c = mag_bits(v.y);
    const unsigned long long h = a > c ? a : c;
    mx = h > mx ? h : mx;
  }
  mx = block_max_u64(mx, sh);
  if (threadIdx.x == 0 && mx != 0) atomicMax(&e[r], exp_bound_bits(mx));
}

// Row slicing: input row r of a complex [rows][K] matrix (leading dimension ld,
// complex units).  form 0: output row r = (x, y)_k; form 1: rows 2r = (x, y)_k
// and 2r+1 = (y, -x)_k.  Q is [S][rows_out_p][Kp] BF16 (padding zeroed), e the
// row exponents (k_oz_rowmax).  grid (input rows incl. padding, ceil(Kp/2 / 2048)).
__global__ void __launch_bounds__(256) k_oz_slice_rows(const double2* __restrict__ src, int ld,
                                                       int rows, int K, int form, int rows_out_p,
                                                       int Kp, const int* __restrict__ e,
                                                       __nv_bfloat16* __restrict__ Q) {
  const int r = blockIdx.x;
  const double2* row = src + (size_t)r * ld;
  const bool valid = r < rows;
  const int ex = valid ? oz_exp(e[r]) : 0;
  const size_t slice2 = (size_t)rows_out_p * Kp / 2;     // one slice, in BF16 pairs
  const int orow = form == 1 ? 2 * r : r;
  unsigned* base0 = reinterpret_cast<unsigned*>(Q + (size_t)orow * Kp);
  unsigned* base1 = reinterpret_cast<unsigned*>(Q + (size_t)(orow + 1) * Kp);
  const int k0 = blockIdx.y * OZ_ROW_CHUNK, k1 = min(Kp / 2, k0 + OZ_ROW_CHUNK);
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (valid && k < K) v = row[k];
    unsigned short qx[OZ_S], qy[OZ_S];
    slices_of(v.x, ex, qx);
    slices_of(v.y, ex, qy);
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) {
      base0[t * slice2 + k] = pack2(qx[t], qy[t]);
      if (form == 1) base1[t * slice2 + k] = pack2(qy[t], (unsigned short)(qx[t] ^ 0x8000u));
    }
  }
}

// Column exponents of a complex [K][M] matrix (leading dimension ld): e[m] for
// max over k of |x|, |y|.  grid (ceil(M / 256), ceil(K / 64)): each thread
// scans 64 rows of its column (consecutive threads, consecutive m) and merges
// its exponent bound with atomicMax (the bound is monotonic in the maximum);
// e must hold 0x80808080 (below every exponent) beforehand, and an all-zero
// column keeps it.
// split: the real and imaginary parts of column m get their own exponents,
// e[2m] and e[2m+1] (the real-K slicing, form 4).
__global__ void k_oz_colmax(const double2* __restrict__ src, int ld, int K, int M, int split,
                            int* __restrict__ e) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int k0 = blockIdx.y * 64, k1 = min(K, k0 + 64);
  unsigned long long mx = 0, my = 0;
#pragma unroll 8
  for (int k = k0; k < k1; ++k) {
    const double2 v = src[(size_t)k * ld + m];
    const unsigned long long a = mag_bits(v.x), c = mag_bits(v.y);
    mx = a > mx ? a : mx;
    my = c > my ? c : my;
  }
  if (split) {
    if (mx != 0) atomicMax(&e[2 * m], exp_bound_bits(mx));
    if (my != 0) atomicMax(&e[2 * m + 1], exp_bound_bits(my));
  } else {
    const unsigned long long h = mx > my ? mx : my;
    if (h != 0) atomicMax(&e[m], exp_bound_bits(h));
  }
}

// Transposed slicing of a complex [K][M] matrix: output rows from its columns.
// form 0: row m = (x, y)_k; form 2: rows 2m = (x, -y)_k and 2m+1 = (y, x)_k
// (K axis of 2K interleaved entries).  Real K axis (K entries, the products
// with a real right-hand matrix): form 4: rows 2m = (x)_k and 2m+1 = (y)_k with
// the exponents e[2m], e[2m+1]; form 5: row m = (x)_k (the real matrix itself).
// 32 x 32 tiles through shared memory (reads coalesced along m, writes along k).
// grid (ceil(cols_p / 32), Kp / 64) with cols_p = the padded column count
// (Kp / 32 for the real forms).
__global__ void k_oz_slice_cols(const double2* __restrict__ src, int ld, int K, int M, int form,
                                const int* __restrict__ e, int rows_out_p, int Kp,
                                __nv_bfloat16* __restrict__ Q) {
  __shared__ double2 tile[32][33];
  const int m0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, m = m0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && m < M) ? src[(size_t)k * ld + m] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const size_t slice = (size_t)rows_out_p * Kp;
  if (form >= 4) {
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int m = m0 + r, k = k0 + threadIdx.x;
      const int orow = form == 4 ? 2 * m : m;
      if (orow >= rows_out_p || k >= Kp) continue;
      const double2 v = tile[threadIdx.x][r];
      unsigned short qx[OZ_S], qy[OZ_S];
      slices_of(v.x, m < M ? oz_exp(e[orow]) : 0, qx);
      unsigned short* p0 = reinterpret_cast<unsigned short*>(Q) + (size_t)orow * Kp + k;
#pragma unroll
      for (int t = 0; t < OZ_S; ++t) p0[t * slice] = qx[t];
      if (form == 4) {
        slices_of(v.y, m < M ? oz_exp(e[orow + 1]) : 0, qy);
#pragma unroll
        for (int t = 0; t < OZ_S; ++t) p0[t * slice + Kp] = qy[t];
      }
    }
    return;
  }
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int m = m0 + r, k = k0 + threadIdx.x;
    const int orow = form == 0 ? m : 2 * m;
    if (orow >= rows_out_p || 2 * k >= Kp) continue;
    const double2 v = tile[threadIdx.x][r];
    const int ex = m < M ? oz_exp(e[m]) : 0;
    unsigned short qx[OZ_S], qy[OZ_S];
    slices_of(v.x, ex, qx);
    slices_of(v.y, ex, qy);
    unsigned* p0 = reinterpret_cast<unsigned*>(Q + (size_t)orow * Kp) + k;
    unsigned* p1 = reinterpret_cast<unsigned*>(Q + (size_t)(orow + 1) * Kp) + k;
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) {
      if (form == 0) {
        p0[t * slice / 2] = pack2(qx[t], qy[t]);
      } else {
        p0[t * slice / 2] = pack2(qx[t], (unsigned short)(qy[t] ^ 0x8000u));
        p1[t * slice / 2] = pack2(qy[t], qx[t]);
      }
    }
  }
}

// Both exponent sets of a complex [R][C] matrix in one read: row r's bound into
// er[r], column c's into ec[c] (both hold 0x80808080 beforehand).  grid
// (ceil(C / 256), ceil(R / 8)), 256 threads: each thread scans 8 rows of one
// column; the row maxima meet through shared memory.
__global__ void __launch_bounds__(256) k_oz_bothmax(const double2* __restrict__ src, int R, int C,
                                                    int* __restrict__ er, int* __restrict__ ec) {
  __shared__ unsigned long long rmax[8][8];   // [row][warp]
  const int cidx = blockIdx.x * 256 + threadIdx.x, r0 = blockIdx.y * 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long cm = 0;
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    const int r = r0 + rr;
    unsigned long long h = 0;
    if (r < R && cidx < C) {
      const double2 v = src[(size_t)r * C + cidx];
      const unsigned long long a = mag_bits(v.x), b = mag_bits(v.y);
      h = a > b ? a : b;
    }
    cm = h > cm ? h : cm;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, h, o);
      h = w > h ? w : h;
    }
    if (lane == 0) rmax[rr][warp] = h;
  }
  if (cidx < C && cm != 0) atomicMax(&ec[cidx], exp_bound_bits(cm));
  __syncthreads();
  if (threadIdx.x < 8 && r0 + threadIdx.x < R) {
    unsigned long long h = 0;
    for (int w = 0; w < 8; ++w) h = rmax[threadIdx.x][w] > h ? rmax[threadIdx.x][w] : h;
    if (h != 0) atomicMax(&er[r0 + threadIdx.x], exp_bound_bits(h));
  }
}

// Both slicings of a complex [R][C] matrix in one read, through 32 x 32 tiles in
// shared memory: Q1 (form 0 of oz_slice_rows: row r = (x, y) over c, exponent
// er[r], [S][rows1][Kp1]) and Q2 (form 0 of oz_slice_cols: row c = (x, y) over
// r, exponent ec[c], [S][rows2][Kp2]), padding zeroed.  grid (ceil(max(C,
// rows2, Kp1/2) / 32), ceil(max(R, rows1, Kp2/2) / 32)), block (32, 8).
__global__ void __launch_bounds__(256) k_oz_slice_both(const double2* __restrict__ src, int R, int C,
                                                       const int* __restrict__ er,
                                                       const int* __restrict__ ec, int rows1, int Kp1,
                                                       unsigned* __restrict__ Q1, int rows2, int Kp2,
                                                       unsigned* __restrict__ Q2) {
  __shared__ double2 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
    const int r = r0 + rr, c = c0 + threadIdx.x;
    tile[rr][threadIdx.x] = (r < R && c < C) ? src[(size_t)r * C + c] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const size_t s1 = (size_t)rows1 * Kp1 / 2, s2 = (size_t)rows2 * Kp2 / 2;
  unsigned short qx[OZ_S], qy[OZ_S];
  // row form: thread (x = c, y) writes rows r0 + y + 8 i, consecutive c along a row
  for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
    const int r = r0 + rr, c = c0 + threadIdx.x;
    if (r >= rows1 || 2 * c >= Kp1) continue;
    const double2 v = tile[rr][threadIdx.x];
    const int ex = r < R ? oz_exp(er[r]) : 0;
    slices_of(v.x, ex, qx);
    slices_of(v.y, ex, qy);
    unsigned* p = Q1 + (size_t)r * (Kp1 / 2) + c;
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) p[t * s1] = pack2(qx[t], qy[t]);
  }
  // column form: thread (x = r, y) writes rows c0 + y + 8 i, consecutive r along a row
  for (int cc = threadIdx.y; cc < 32; cc += blockDim.y) {
    const int c = c0 + cc, r = r0 + threadIdx.x;
    if (c >= rows2 || 2 * r >= Kp2) continue;
    const double2 v = tile[threadIdx.x][cc];
    const int ex = c < C ? oz_exp(ec[c]) : 0;
    slices_of(v.x, ex, qx);
    slices_of(v.y, ex, qy);
    unsigned* p = Q2 + (size_t)c * (Kp2 / 2) + r;
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) p[t * s2] = pack2(qx[t], qy[t]);
  }
}

// P[m][n] = sum_z part[z][n][m] (fixed order), into C with leading dimension ldc.
__global__ void k_oz_reduce(const double2* __restrict__ part, int nsplit, long long zstride,
                            int Mp, int M, int N, double2* __restrict__ C, int ldc) {
  const size_t total = (size_t)M * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / N), n = (int)(i % N);
    double sx = 0.0, sy = 0.0;
    for (int z = 0; z < nsplit; ++z) {
      const double2 v = part[(size_t)z * zstride + (size_t)n * Mp + m];
      sx += v.x;
      sy += v.y;
    }
    C[(size_t)m * ldc + n] = make_double2(sx, sy);
  }
}

// The real-output form: part[z][p][m] holds (Re C[m][2p], Re C[m][2p+1]);
// C[m][n] = (sum_z, 0) for n < N, fixed order.
__global__ void k_oz_reduce_real(const double2* __restrict__ part, int nsplit, long long zstride,
                                 int Mp, int M, int N, double2* __restrict__ C, int ldc) {
  const int np = (N + 1) / 2;
  const size_t total = (size_t)M * np;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / np), p = (int)(i % np);
    double sx = 0.0, sy = 0.0;
    for (int z = 0; z < nsplit; ++z) {
      const double2 v = part[(size_t)z * zstride + (size_t)p * Mp + m];
      sx += v.x;
      sy += v.y;
    }
    C[(size_t)m * ldc + 2 * p] = make_double2(sx, 0.0);
    if (2 * p + 1 < N) C[(size_t)m * ldc + 2 * p + 1] = make_double2(sy, 0.0);
  }
}

// ---- host side ----------------------------------------------------------------
static inline int pad_to(int x, int m) { return (x + m - 1) / m * m; }
static inline size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

static int oz_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QE_ECUDA;
  }
  return QE_OK;
}

// rows x Kp BF16 matrix, K-major, box `box_rows` rows x 64 columns, 128-byte swizzle.
static int oz_map(CUtensorMap* m, const __nv_bfloat16* ptr, int rows, int Kp, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  int rc = tc_get_encode(&enc);
  if (rc) return rc;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)ptr, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (BF16) failed (%d)", (int)r);
    return QE_ECUDA;
  }
  return QE_OK;
}

// Sliced operand: S slices of a [rows_p][Kp] BF16 matrix and its row exponents.
struct OzOperand {
  __nv_bfloat16* q = nullptr;
  int* e = nullptr;
  int rows_p = 0, Kp = 0;   // the allocation: [S][rows_p][Kp]
  int rows_used = 0;        // rows the products tile (<= rows_p, a multiple of 128)
};

size_t oz_operand_bytes(int rows_out, int K) {
  const size_t rp = pad_to(std::max(rows_out, 1), OZ_BM), kp = pad_to(2 * std::max(K, 1), OZ_BK);
  return up256((size_t)OZ_S * rp * kp * 2) + up256(rp * sizeof(int)) + 256;
}

static OzOperand oz_carve(void* mem, int rows_out, int K) {
  OzOperand o;
  o.rows_p = pad_to(std::max(rows_out, 1), OZ_BM);
  o.rows_used = o.rows_p;
  o.Kp = pad_to(2 * std::max(K, 1), OZ_BK);
  char* p = reinterpret_cast<char*>(((uintptr_t)mem + 255) & ~(uintptr_t)255);
  o.q = reinterpret_cast<__nv_bfloat16*>(p);
  o.e = reinterpret_cast<int*>(p + up256((size_t)OZ_S * o.rows_p * o.Kp * 2));
  return o;
}

// Slices of the rows of a complex [rows][K] matrix (form 0: one output row per
// input row, also the B operand of the real-output inner product; form 1: the
// inner product's B pair).  Returns the carved operand.
int oz_slice_rows(const double* src, int ld, int rows, int K, int form, void* mem, OzOperand* out,
                  cudaStream_t st, Prof* pf) {
  const int rows_out = form == 1 ? 2 * rows : rows;
  *out = oz_carve(mem, rows_out, K);
  if (rows > 0) {
    ProfScope ps(pf, "k_oz_rowmax", st);
    // padding rows too: the real-output product reads the exponent of the
    // ragged last column pair's empty half
    if (cudaMemsetAsync(out->e, 0x80, (size_t)out->rows_p * sizeof(int), st) != cudaSuccess) {
      set_error("oz_slice_rows: memset failed");
      return QE_ECUDA;
    }
    dim3 gm(rows, (K + OZ_ROW_CHUNK - 1) / OZ_ROW_CHUNK);
    k_oz_rowmax<<<gm, 256, 0, st>>>(reinterpret_cast<const double2*>(src), ld, K, out->e);
    int rc = oz_check("k_oz_rowmax");
    if (rc) return rc;
  }
  ProfScope ps(pf, "k_oz_slice_rows", st);
  const int in_rows_p = form == 1 ? out->rows_p / 2 : out->rows_p;
  dim3 g(in_rows_p, (out->Kp / 2 + OZ_ROW_CHUNK - 1) / OZ_ROW_CHUNK);
  k_oz_slice_rows<<<g, 256, 0, st>>>(reinterpret_cast<const double2*>(src), ld, rows, K, form,
                                     out->rows_p, out->Kp, out->e, out->q);
  return oz_check("k_oz_slice_rows");
}

// Slices of the columns of a complex [K][cols] matrix (form 0: one output row
// per column; form 2: the outer product's B pair).
int oz_slice_cols(const double* src, int ld, int K, int cols, int form, void* mem, OzOperand* out,
                  cudaStream_t st, Prof* pf) {
  const bool real_k = form >= 4;
  const int rows_out = (form == 0 || form == 5) ? cols : 2 * cols;
  *out = oz_carve(mem, rows_out, real_k ? (K + 1) / 2 : K);
  {
    ProfScope ps(pf, "k_oz_colmax", st);
    if (cudaMemsetAsync(out->e, 0x80, (size_t)out->rows_p * sizeof(int), st) != cudaSuccess) {
      set_error("oz_slice_cols: memset failed");
      return QE_ECUDA;
    }
    dim3 gm((cols + 255) / 256, (K + 63) / 64);
    k_oz_colmax<<<gm, 256, 0, st>>>(reinterpret_cast<const double2*>(src), ld, K, cols,
                                    form == 4 ? 1 : 0, out->e);
    int rc = oz_check("k_oz_colmax");
    if (rc) return rc;
  }
  ProfScope ps(pf, "k_oz_slice_cols", st);
  const int cols_p = rows_out == cols ? out->rows_p : out->rows_p / 2;
  dim3 g((cols_p + 31) / 32, real_k ? out->Kp / 32 : out->Kp / 64);
  k_oz_slice_cols<<<g, dim3(32, 8), 0, st>>>(reinterpret_cast<const double2*>(src), ld, K, cols,
                                             form, out->e, out->rows_p, out->Kp, out->q);
  return oz_check("k_oz_slice_cols");
}

// Both slicings of a complex [R][C] matrix (ld = C) from one max pass and one
// slicing pass: *rows = oz_slice_rows(form 0) into mem1, *cols =
// oz_slice_cols(form 0) into mem2 -- the same operands, bit for bit.
int oz_slice_both(const double* src, int R, int C, void* mem1, void* mem2, OzOperand* rows,
                  OzOperand* cols, cudaStream_t st, Prof* pf) {
  *rows = oz_carve(mem1, R, C);
  *cols = oz_carve(mem2, C, R);
  {
    ProfScope ps(pf, "k_oz_bothmax", st);
    if (cudaMemsetAsync(rows->e, 0x80, (size_t)rows->rows_p * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(cols->e, 0x80, (size_t)cols->rows_p * sizeof(int), st) != cudaSuccess) {
      set_error("oz_slice_both: memset failed");
      return QE_ECUDA;
    }
    k_oz_bothmax<<<dim3((C + 255) / 256, (R + 7) / 8), 256, 0, st>>>(
        reinterpret_cast<const double2*>(src), R, C, rows->e, cols->e);
    int rc = oz_check("k_oz_bothmax");
    if (rc) return rc;
  }
  ProfScope ps(pf, "k_oz_slice_both", st);
  const int cx = std::max(C, std::max(cols->rows_p, rows->Kp / 2));
  const int ry = std::max(R, std::max(rows->rows_p, cols->Kp / 2));
  k_oz_slice_both<<<dim3((cx + 31) / 32, (ry + 31) / 32), dim3(32, 8), 0, st>>>(
      reinterpret_cast<const double2*>(src), R, C, rows->e, cols->e, rows->rows_p, rows->Kp,
      reinterpret_cast<unsigned*>(rows->q), cols->rows_p, cols->Kp, reinterpret_cast<unsigned*>(cols->q));
  return oz_check("k_oz_slice_both");
}

// ---- projectors generated on the fly, straight into the slices -------------------
// One thread per (atom, plane wave) forms the atom's structure factor once,
//   S = e^{-i k.R} T_x[m_x] T_y[m_y] T_z[m_z],   T_c[m] = e^{-i 2 pi m f_c},
// and from it every projector of the atom, beta = S (-i)^l Y_lc(q) F_n(G),
// which it cuts into the row slices (inner product: row = projector) and the
// column slices (outer product: row = plane wave) at once.  No beta array is
// read or written.  The exponents come from bounds that do not depend on the
// atom (|S| = 1): per projector component, max over G of |Y_lc(q) F_n(G)|; per
// plane wave, the max over the components; each times (1 + 2^-40), which covers
// the rounding of S, so that every sliced value is below 2^e.
__device__ __forceinline__ void gen_q(const GenProj& g, int G, double q[3]) {
  const int m0 = g.mill[3 * G], m1 = g.mill[3 * G + 1], m2 = g.mill[3 * G + 2];
#pragma unroll
  for (int c = 0; c < 3; ++c) q[c] = ((g.k[c] + m0 * g.b[c]) + m1 * g.b[3 + c]) + m2 * g.b[6 + c];
}

// |Y_lc(q)| F_n(G) (the magnitude of every projector component at G)
__device__ __forceinline__ double gen_amp(const GenProj& g, int n, int c, int G, const double q[3]) {
  const double f = fabs(g.radial[(size_t)n * g.npw + G]);
  if (g.l[n] == 0) return 0.28209479177387814347 * f;           // 1 / (2 sqrt(pi))
  return 0.48860251190291992159 * fabs(q[c]) * f;                // sqrt(3 / (4 pi)) |q_c|
}

// Exponent bounds.  grid (ceil(npw / 256), 1): per-G column exponents, and the
// per-component maxima merged with atomicMax (as ordered bit patterns) into cmax.
__global__ void k_gen_exps(GenProj g, unsigned long long* __restrict__ cmax, int* __restrict__ ecol,
                           int form4) {
  const int G = blockIdx.x * blockDim.x + threadIdx.x;
  if (G >= g.npw) return;
  double q[3];
  gen_q(g, G, q);
  double mx = 0.0;
  int j = 0;
  for (int n = 0; n < g.nrad; ++n)
    for (int c = 0; c < 2 * g.l[n] + 1; ++c, ++j) {
      const double a = gen_amp(g, n, c, G, q);
      mx = fmax(mx, a);
      atomicMax(&cmax[j], mag_bits(a));
    }
  const int ex = mx > 0.0 ? exp_bound(mx * (1.0 + 0x1p-40)) : (int)0x80808080;
  if (form4) {   // |Re beta|, |Im beta| <= |beta|: the bound of both rows of G
    ecol[2 * G] = ex;
    ecol[2 * G + 1] = ex;
  } else {
    ecol[G] = ex;
  }
}

// Row exponents of every projector from the component maxima.
__global__ void k_gen_erow(GenProj g, const unsigned long long* __restrict__ cmax, int* __restrict__ erow) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.np) return;
  const double a = __longlong_as_double((long long)cmax[i % g.nper]);
  erow[i] = a > 0.0 ? exp_bound(a * (1.0 + 0x1p-40)) : (int)0x80808080;
}

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// beta of atom I at plane wave G for every projector of the atom, handed to f(i, beta)
template <typename F>
__device__ __forceinline__ void gen_atom(const GenProj& g, int I, int G, F&& f) {
  double q[3];
  gen_q(g, G, q);
  const double2* tab = reinterpret_cast<const double2*>(g.tab) + (size_t)I * g.tstride;
  const int m0 = g.mill[3 * G], m1 = g.mill[3 * G + 1], m2 = g.mill[3 * G + 2];
  double2 S = reinterpret_cast<const double2*>(g.ekr)[I];
  S = cmul2(S, tab[g.toff[0] + m0 + g.half[0]]);
  S = cmul2(S, tab[g.toff[1] + m1 + g.half[1]]);
  S = cmul2(S, tab[g.toff[2] + m2 + g.half[2]]);
  for (int n = 0; n < g.nrad; ++n) {
    const double rad = g.radial[(size_t)n * g.npw + G];
    if (g.l[n] == 0) {
      const double a = 0.28209479177387814347 * rad;
      f(I * g.nper + g.off[n], make_double2(S.x * a, S.y * a));
    } else {
      for (int c = 0; c < 3; ++c) {
        const double a = 0.48860251190291992159 * q[c] * rad;
        f(I * g.nper + g.off[n] + c, make_double2(S.y * a, -S.x * a));   // (-i) S a
      }
    }
  }
}

// Both slicings.  grid (ceil(npw / 128), natom); A1: [S][rows_p1][Kp1] (row i,
// K pair (2G, 2G+1)); A2: [S][rows_p2][Kp2] (row G, K pair (2i, 2i+1)).  The A1
// words of a projector are consecutive in G, so consecutive threads store them
// together; the A2 words of one G are the atom's nper consecutive columns, which
// one thread produces one projector at a time -- they are staged in shared
// memory (sQ[t][g][j], 8 x 128 x nper words) and stored row by row, a warp
// writing whole 32-byte sectors instead of 4-byte pieces.
__global__ void __launch_bounds__(128) k_gen_slices(GenProj g, const int* __restrict__ erow,
                                                    const int* __restrict__ ecol, int rows_p1, int Kp1,
                                                    unsigned* __restrict__ Q1, int rows_p2, int Kp2,
                                                    unsigned* __restrict__ Q2, int form4) {
  extern __shared__ unsigned sQ[];
  const int G0 = blockIdx.x * blockDim.x, G = G0 + threadIdx.x, I = blockIdx.y;
  const int nper = g.nper, nt = blockDim.x;
  const size_t s1 = (size_t)rows_p1 * Kp1 / 2, s2 = (size_t)rows_p2 * Kp2 / 2;
  if (G < g.npw) {
    const int ec = oz_exp(ecol[form4 ? 2 * G : G]);
    gen_atom(g, I, G, [&](int i, double2 v) {
      unsigned short qx[OZ_S], qy[OZ_S];
      const int er = oz_exp(erow[i]);
      slices_of(v.x, er, qx);
      slices_of(v.y, er, qy);
      unsigned* p1 = Q1 + (size_t)i * (Kp1 / 2) + G;
#pragma unroll
      for (int t = 0; t < OZ_S; ++t) p1[t * s1] = pack2(qx[t], qy[t]);
      slices_of(v.x, ec, qx);
      slices_of(v.y, ec, qy);
      const int j = i - I * nper;
#pragma unroll
      for (int t = 0; t < OZ_S; ++t) sQ[((size_t)t * nt + threadIdx.x) * nper + j] = pack2(qx[t], qy[t]);
    });
  }
  __syncthreads();
  const int rows = min(nt, g.npw - G0);
  const int per_t = rows * nper;
  if (form4) {
    // real K axis: row 2G the real parts, row 2G+1 the imaginary parts (BF16 each)
    unsigned short* Qu = reinterpret_cast<unsigned short*>(Q2);
    const size_t su = (size_t)rows_p2 * Kp2;
    for (int w = threadIdx.x; w < OZ_S * per_t; w += nt) {
      const int t = w / per_t, r = w - t * per_t;
      const int gg = r / nper, j = r - gg * nper;
      const unsigned v = sQ[((size_t)t * nt + gg) * nper + j];
      unsigned short* q = Qu + t * su + (size_t)(2 * (G0 + gg)) * Kp2 + (size_t)I * nper + j;
      q[0] = (unsigned short)(v & 0xFFFFu);
      q[Kp2] = (unsigned short)(v >> 16);
    }
    return;
  }
  for (int w = threadIdx.x; w < OZ_S * per_t; w += nt) {
    const int t = w / per_t, r = w - t * per_t;
    const int gg = r / nper, j = r - gg * nper;
    Q2[t * s2 + (size_t)(G0 + gg) * (Kp2 / 2) + (size_t)I * nper + j] =
        sQ[((size_t)t * nt + gg) * nper + j];
  }
}

// Zero the rectangle [r0, r1) x [c0, c1) (uint32 units) of every slice.
__global__ void k_zero_rect(unsigned* __restrict__ Q, size_t slice, int ld, int r0, int r1, int c0,
                            int c1) {
  const size_t w = (size_t)(c1 - c0), total = (size_t)(r1 - r0) * w * OZ_S;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t s = t / ((size_t)(r1 - r0) * w), rem = t % ((size_t)(r1 - r0) * w);
    const int r = r0 + (int)(rem / w), c = c0 + (int)(rem % w);
    Q[s * slice + (size_t)r * ld + c] = 0u;
  }
}

static int zero_rect(unsigned* Q, size_t slice, int ld, int r0, int r1, int c0, int c1, cudaStream_t st) {
  if (r1 <= r0 || c1 <= c0) return QE_OK;
  const size_t total = (size_t)(r1 - r0) * (c1 - c0) * OZ_S;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 8);
  k_zero_rect<<<blocks, 256, 0, st>>>(Q, slice, ld, r0, r1, c0, c1);
  return oz_check("k_zero_rect");
}

size_t oz_gen_scratch_bytes(const GenProj& g) {
  return up256((size_t)g.nper * sizeof(unsigned long long)) + 256;
}

int oz_gen_beta(const GenProj& g, void* bslices, void* scratch, cudaStream_t st, Prof* pf, bool form4) {
  if (g.np <= 0 || g.npw <= 0) return QE_OK;
  if (form4 && g.np % 2 != 0) {
    set_error("oz_gen_beta: the real-K column form needs an even projector count");
    return QE_EINVAL;
  }
  char* bs = static_cast<char*>(bslices);
  const OzOperand A1 = oz_carve(bs, g.np, g.npw);
  const OzOperand A2 = form4 ? oz_carve(bs + oz_operand_bytes(g.np, g.npw), 2 * g.npw, g.np / 2)
                             : oz_carve(bs + oz_operand_bytes(g.np, g.npw), g.npw, g.np);
  unsigned long long* cmax = static_cast<unsigned long long*>(scratch);
  ProfScope ps(pf, "k_gen_slices", st);
  if (cudaMemsetAsync(cmax, 0, (size_t)g.nper * sizeof(unsigned long long), st) != cudaSuccess) {
    set_error("oz_gen_beta: memset failed");
    return QE_ECUDA;
  }
  k_gen_exps<<<(g.npw + 255) / 256, 256, 0, st>>>(g, cmax, A2.e, form4 ? 1 : 0);
  k_gen_erow<<<(g.np + 255) / 256, 256, 0, st>>>(g, cmax, A1.e);
  int rc = oz_check("k_gen_exps");
  if (rc) return rc;
  unsigned* Q1 = reinterpret_cast<unsigned*>(A1.q);
  unsigned* Q2 = reinterpret_cast<unsigned*>(A2.q);
  const size_t s1 = (size_t)A1.rows_p * A1.Kp / 2, s2 = (size_t)A2.rows_p * A2.Kp / 2;
  // the padding of both slicings (uint32 words: pairs of BF16), then the values
  const int rows2 = form4 ? 2 * g.npw : g.npw, cols2 = form4 ? g.np / 2 : g.np;
  if ((rc = zero_rect(Q1, s1, A1.Kp / 2, g.np, A1.rows_p, 0, A1.Kp / 2, st)) ||
      (rc = zero_rect(Q1, s1, A1.Kp / 2, 0, g.np, g.npw, A1.Kp / 2, st)) ||
      (rc = zero_rect(Q2, s2, A2.Kp / 2, rows2, A2.rows_p, 0, A2.Kp / 2, st)) ||
      (rc = zero_rect(Q2, s2, A2.Kp / 2, 0, rows2, cols2, A2.Kp / 2, st)))
    return rc;
  const size_t gsm = (size_t)OZ_S * 128 * g.nper * sizeof(unsigned);   // <= 96 KB (nper <= 24)
  set_max_dynamic_smem(k_gen_slices);
  k_gen_slices<<<dim3((g.npw + 127) / 128, g.natom), 128, gsm, st>>>(g, A1.e, A2.e, A1.rows_p, A1.Kp,
                                                                      Q1, A2.rows_p, A2.Kp, Q2,
                                                                      form4 ? 1 : 0);
  if (pf) pf->launches += 6;
  return oz_check("k_gen_slices");
}

// The generated beta as values (row i = projector, complex [np][npw]).
__global__ void __launch_bounds__(128) k_gen_values(GenProj g, double2* __restrict__ beta) {
  const int G = blockIdx.x * blockDim.x + threadIdx.x, I = blockIdx.y;
  if (G >= g.npw) return;
  gen_atom(g, I, G, [&](int i, double2 v) { beta[(size_t)i * g.npw + G] = v; });
}

int gen_beta_values(const GenProj& g, double* beta, cudaStream_t st, Prof* pf) {
  if (g.np <= 0 || g.npw <= 0) return QE_OK;
  ProfScope ps(pf, "k_gen_values", st);
  k_gen_values<<<dim3((g.npw + 127) / 128, g.natom), 128, 0, st>>>(g, reinterpret_cast<double2*>(beta));
  return oz_check("k_gen_values");
}

// K splits: as many CTAs as fit in ONE wave (one CTA per SM: the kernel holds
// all of TMEM and ~195 KB of shared memory), at least one chunk each.
static int oz_splits(int tiles, int nks) {
  int ns = std::max(1, 152 / std::max(1, tiles));
  ns = std::min(ns, std::max(1, nks / OZ_KPC));   // at least one full chunk per CTA
  const int per = (nks + ns - 1) / ns;
  return (nks + per - 1) / per;
}

// Partials of the complex inner product (2N GEMM columns) or of its real-output
// form (N columns, fewer tiles, so possibly more K splits): the larger of the two.
size_t oz_partial_bytes(int M, int N, int K) {
  const int Mp = pad_to(std::max(M, 1), OZ_BM);
  const int nks = pad_to(2 * std::max(K, 1), OZ_BK) / OZ_BK;
  size_t b = 0;
  for (int cols : {2 * std::max(N, 1), std::max(N, 1)}) {
    const int Np = pad_to(cols, OZ_BM);
    const int ns = oz_splits((Mp / OZ_BM) * (Np / OZ_BN), nks);
    b = std::max(b, (size_t)ns * (Np / 2) * Mp * 16);
  }
  return up256(b);
}

static int oz_launch(const OzOperand& A, const OzOperand& B, int M, int N, double2* out, int ldo,
                     long long zstride, int nsplit, int alpha_neg, int beta, int ecol,
                     int* status, cudaStream_t st, Prof* pf) {
  if (A.Kp != B.Kp) {
    set_error("oz_gemm: K padding mismatch");
    return QE_EINVAL;
  }
  CUtensorMap mA, mB;
  int rc;
  if ((rc = oz_map(&mA, A.q, OZ_S * A.rows_p, A.Kp, OZ_BM)) ||
      (rc = oz_map(&mB, B.q, OZ_S * B.rows_p, B.Kp, OZ_BN)))
    return rc;
  const int nks = A.Kp / OZ_BK;
  const int per = (nks + nsplit - 1) / nsplit;
  set_max_dynamic_smem(k_oz_gemm);
  ProfScope ps(pf, "k_oz_gemm", st);
  dim3 g(B.rows_p / OZ_BN, A.rows_used / OZ_BM, nsplit);
  k_oz_gemm<<<g, OZ_THREADS, OZ_SMEM_BYTES, st>>>(mA, mB, A.rows_p, B.rows_p, nks, per, A.e, B.e,
                                                   out, ldo, zstride, M, N, alpha_neg, beta, ecol,
                                                   status);
  return oz_check("k_oz_gemm");
}

// C[m][n] = sum_k conj(A[m][k]) B[n][k] with A sliced by oz_slice_rows (form 0)
// and B by oz_slice_rows (form 1); split K, fixed-order reduction.  real: C[m][n]
// = (Re sum_k conj(A[m][k]) B[n][k], 0) with B sliced in form 0, so that the
// GEMM's column pair (2p, 2p+1) holds the real parts of the complex columns 2p
// and 2p+1, each scaled by its own row's exponent: half the columns of the
// complex form.
int oz_gemm_inner(const OzOperand& A, const OzOperand& B, int M, int N, double* C, int ldc,
                  void* part, size_t part_bytes, int* status, cudaStream_t st, Prof* pf,
                  bool real = false) {
  if (M <= 0 || N <= 0) return QE_OK;
  const int Nc = N;
  if (real) N = (N + 1) / 2;   // GEMM column pairs
  const int nks = A.Kp / OZ_BK;
  int ns = oz_splits((A.rows_used / OZ_BM) * (B.rows_p / OZ_BN), nks);
  const long long zstride = (long long)(B.rows_p / 2) * A.rows_used;
  const size_t cap = part_bytes / ((size_t)zstride * 16);   // splits the buffer holds
  if (cap < 1) {
    set_error("oz_gemm_inner: partial buffer too small");
    return QE_EINVAL;
  }
  if ((size_t)ns > cap) {   // fewer, longer K ranges (none empty)
    const int per = (nks + (int)cap - 1) / (int)cap;
    ns = (nks + per - 1) / per;
  }
  int rc = oz_launch(A, B, M, N, reinterpret_cast<double2*>(part), A.rows_used, zstride, ns, 0, 0,
                     real ? 1 : 0, status, st, pf);
  if (rc) return rc;
  const int per = (nks + ns - 1) / ns;
  const int nsplit = (nks + per - 1) / per;
  ProfScope ps(pf, "k_oz_reduce", st);
  const size_t total = (size_t)M * N;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 8);
  if (real)
    k_oz_reduce_real<<<blocks, 256, 0, st>>>(reinterpret_cast<const double2*>(part), nsplit,
                                             zstride, A.rows_used, M, Nc,
                                             reinterpret_cast<double2*>(C), ldc);
  else
    k_oz_reduce<<<blocks, 256, 0, st>>>(reinterpret_cast<const double2*>(part), nsplit, zstride,
                                        A.rows_used, M, N, reinterpret_cast<double2*>(C), ldc);
  return oz_check("k_oz_reduce");
}

// C[n][m] (+)= (-) sum_k A[k][m] B[k][n] with A sliced by oz_slice_cols (form 0)
// and B by oz_slice_cols (form 2).
int oz_gemm_outer(const OzOperand& A, const OzOperand& B, int M, int N, double* C, int ldc,
                  int alpha_neg, int beta, int* status, cudaStream_t st, Prof* pf) {
  if (M <= 0 || N <= 0) return QE_OK;
  return oz_launch(A, B, M, N, reinterpret_cast<double2*>(C), ldc, 0, 1, alpha_neg, beta, 0,
                   status, st, pf);
}

bool fp64_gemm_on_tensor_cores() {
  static const bool on = [] {
    const char* v = std::getenv("QE_FP64_GEMM");
    return !(v && std::strcmp(v, "simt") == 0);
  }();
  return on;
}

// Whether an FP64 complex product of this size goes to the tensor cores: the
// slicing launches and the one-wave split cost ~30 us, which the DFMA kernels
// recover below ~4 M complex multiply-adds.
bool oz_worth(long long M, long long N, long long K) {
  return fp64_gemm_on_tensor_cores() && M > 0 && N > 0 && M * N * K >= (1ll << 22);
}

// ---- general complex products from FP64 operands ------------------------------------
size_t oz_inner_scratch(int M, int N, int K) {
  if (M <= 0 || N <= 0) return 0;
  return oz_operand_bytes(M, K) + oz_operand_bytes(2 * N, K) + oz_partial_bytes(M, N, K);
}

size_t oz_outer_scratch(int M, int N, int K) {
  if (M <= 0 || N <= 0) return 0;
  return oz_operand_bytes(M, K) + oz_operand_bytes(2 * N, K);
}

// C[m][n] = sum_k conj(A[m][k]) B[n][k] (rows of A and B contiguous in k,
// leading dimensions in complex units), FP64-accurate on the tensor cores;
// real: C[m][n] = (Re of it, 0) at half the tensor-core work.
int oz_inner(const double* A, int lda, const double* B, int ldb, int M, int N, int K, double* C,
             int ldc, void* scratch, size_t scratch_bytes, int* status, cudaStream_t st, Prof* pf,
             bool real) {
  if (M <= 0 || N <= 0) return QE_OK;
  if (oz_inner_scratch(M, N, K) > scratch_bytes) {
    set_error("oz_inner: scratch too small");
    return QE_EINVAL;
  }
  char* p = static_cast<char*>(scratch);
  OzOperand a, b;
  int rc;
  if ((rc = oz_slice_rows(A, lda, M, K, 0, p, &a, st, pf))) return rc;
  p += oz_operand_bytes(M, K);
  if ((rc = oz_slice_rows(B, ldb, N, K, real ? 0 : 1, p, &b, st, pf))) return rc;
  p += oz_operand_bytes(2 * N, K);
  return oz_gemm_inner(a, b, M, N, C, ldc, p, oz_partial_bytes(M, N, K), status, st, pf, real);
}

// C[n][m] (+)= (-) sum_k A[k][m] B[k][n] (rows of A and B indexed by k),
// FP64-accurate on the tensor cores.
int oz_outer(const double* A, int lda, const double* B, int ldb, int M, int N, int K, double* C,
             int ldc, int alpha_neg, int beta, void* scratch, size_t scratch_bytes, int* status,
             cudaStream_t st, Prof* pf) {
  if (M <= 0 || N <= 0) return QE_OK;
  if (oz_outer_scratch(M, N, K) > scratch_bytes) {
    set_error("oz_outer: scratch too small");
    return QE_EINVAL;
  }
  char* p = static_cast<char*>(scratch);
  OzOperand a, b;
  int rc;
  if ((rc = oz_slice_cols(A, lda, K, M, 0, p, &a, st, pf))) return rc;
  p += oz_operand_bytes(M, K);
  if ((rc = oz_slice_cols(B, ldb, K, N, 2, p, &b, st, pf))) return rc;
  return oz_gemm_outer(a, b, M, N, C, ldc, alpha_neg, beta, status, st, pf);
}

// C[n][m] (+)= (-) sum_k A[k][m] Re B[k][n] (B real, its imaginary parts not
// read): A's columns sliced as separate real and imaginary rows over a real K
// axis (form 4), B's columns as real rows (form 5), so the GEMM has 2M rows, N
// columns and depth K -- half the tensor-core work of the complex form, whose
// B pair rows would carry the zero imaginary parts.
size_t oz_outer_real_scratch(int M, int N, int K) {
  if (M <= 0 || N <= 0) return 0;
  const int kc = (K + 1) / 2;
  return oz_operand_bytes(2 * M, kc) + oz_operand_bytes(N, kc);
}

int oz_outer_real(const double* A, int lda, const double* B, int ldb, int M, int N, int K,
                  double* C, int ldc, int alpha_neg, int beta, void* scratch, size_t scratch_bytes,
                  int* status, cudaStream_t st, Prof* pf) {
  if (M <= 0 || N <= 0) return QE_OK;
  if (oz_outer_real_scratch(M, N, K) > scratch_bytes) {
    set_error("oz_outer_real: scratch too small");
    return QE_EINVAL;
  }
  char* p = static_cast<char*>(scratch);
  OzOperand a, b;
  int rc;
  if ((rc = oz_slice_cols(A, lda, K, M, 4, p, &a, st, pf))) return rc;
  p += oz_operand_bytes(2 * M, (K + 1) / 2);
  if ((rc = oz_slice_cols(B, ldb, K, N, 5, p, &b, st, pf))) return rc;
  return oz_launch(a, b, 2 * M, N, reinterpret_cast<double2*>(C), ldc, 0, 1, alpha_neg, beta, 2,
                   status, st, pf);
}

// ---- row slices kept across products -------------------------------------------
// A matrix whose rows are only ever appended (the Davidson basis) keeps its row
// slices in `mem` ([S][pad(rows_cap)][Kp], per-row exponents): rows are sliced
// once, when they are added, and the inner products with its first M rows tile
// only pad(M) of them.  Rows past M in the last tile may hold older slices; a
// product row depends on its own A row only, and rows past M are never written.
size_t oz_cache_bytes(int rows_cap, int K) { return oz_operand_bytes(rows_cap, K); }

int oz_cache_rows(const double* src, int ld, int r0, int r1, int K, int rows_cap, void* mem,
                  cudaStream_t st, Prof* pf) {
  if (r1 <= r0) return QE_OK;
  if (r0 < 0 || r1 > rows_cap) {
    set_error("oz_cache_rows: rows [%d, %d) outside the cache of %d", r0, r1, rows_cap);
    return QE_EINVAL;
  }
  const OzOperand o = oz_carve(mem, rows_cap, K);
  const int n = r1 - r0;
  const double2* s2 = reinterpret_cast<const double2*>(src) + (size_t)r0 * ld;
  {
    ProfScope ps(pf, "k_oz_rowmax", st);
    if (cudaMemsetAsync(o.e + r0, 0x80, (size_t)n * sizeof(int), st) != cudaSuccess) {
      set_error("oz_cache_rows: memset failed");
      return QE_ECUDA;
    }
    k_oz_rowmax<<<dim3(n, (K + OZ_ROW_CHUNK - 1) / OZ_ROW_CHUNK), 256, 0, st>>>(s2, ld, K, o.e + r0);
    int rc = oz_check("k_oz_rowmax");
    if (rc) return rc;
  }
  ProfScope ps(pf, "k_oz_slice_rows", st);
  k_oz_slice_rows<<<dim3(n, (o.Kp / 2 + OZ_ROW_CHUNK - 1) / OZ_ROW_CHUNK), 256, 0, st>>>(
      s2, ld, n, K, 0, o.rows_p, o.Kp, o.e + r0, o.q + (size_t)r0 * o.Kp);
  return oz_check("k_oz_slice_rows");
}

size_t oz_inner_cached_scratch(int M, int N, int K) {
  if (M <= 0 || N <= 0) return 0;
  return oz_operand_bytes(2 * N, K) + oz_partial_bytes(M, N, K);
}

// oz_inner with A = the first M rows kept in `mem` (oz_cache_rows).
int oz_inner_cached(const void* mem, int rows_cap, int M, const double* B, int ldb, int N, int K,
                    double* C, int ldc, void* scratch, size_t scratch_bytes, int* status,
                    cudaStream_t st, Prof* pf, bool real) {
  if (M <= 0 || N <= 0) return QE_OK;
  if (M > rows_cap || oz_inner_cached_scratch(M, N, K) > scratch_bytes) {
    set_error("oz_inner_cached: %d rows of %d, or scratch too small", M, rows_cap);
    return QE_EINVAL;
  }
  OzOperand a = oz_carve(const_cast<void*>(mem), rows_cap, K);
  a.rows_used = pad_to(M, OZ_BM);
  char* p = static_cast<char*>(scratch);
  OzOperand b;
  int rc;
  if ((rc = oz_slice_rows(B, ldb, N, K, real ? 0 : 1, p, &b, st, pf))) return rc;
  p += oz_operand_bytes(2 * N, K);
  return oz_gemm_inner(a, b, M, N, C, ldc, p, oz_partial_bytes(M, N, K), status, st, pf, real);
}

// ---- the nonlocal term -----------------------------------------------------------
bool nonlocal_oz_real_outer(bool real_p, int np) { return real_p && np % 2 == 0; }

size_t nonlocal_oz_beta_bytes(int np, int npw) {
  return oz_operand_bytes(np, npw) +
         std::max(oz_operand_bytes(npw, np), oz_operand_bytes(2 * npw, (np + 1) / 2));
}

size_t nonlocal_oz_bytes(int np, int nb, int npw) {
  return oz_operand_bytes(2 * nb, npw) + oz_partial_bytes(np, nb, npw) +
         oz_operand_bytes(2 * nb, np) + 2 * up256((size_t)np * nb * 16) + 1024;
}

// hpsi += beta^T D (conj(beta) psi^T) with FP64-accurate products on the BF16
// tensor cores.  bslices (nonlocal_oz_beta_bytes) holds the two slicings of
// beta (rows for the inner product, columns for the outer one); they are
// (re)computed when slice_beta is true.
int nonlocal_oz(const double* beta, const double* dmat, const double* psi, double* hpsi, int np,
                int nb, int npw, void* bslices, bool slice_beta, void* work, size_t work_bytes,
                int* status, cudaStream_t st, Prof* pf, bool real_p) {
  if (np <= 0 || nb <= 0) return QE_OK;
  if (nonlocal_oz_bytes(np, nb, npw) > work_bytes) {
    set_error("nonlocal_oz: workspace too small");
    return QE_EINVAL;
  }
  char* bs = static_cast<char*>(bslices);
  OzOperand A1, A2, B1, B2;
  int rc;
  // real_p: Q = D Re P is real, so the outer product takes beta's columns as
  // separate real and imaginary rows over a real K axis (half the work)
  const bool r4 = nonlocal_oz_real_outer(real_p, np);
  if (slice_beta && !r4) {
    // both forms from one max pass and one slicing pass over beta
    if ((rc = oz_slice_both(beta, np, npw, bs, bs + oz_operand_bytes(np, npw), &A1, &A2, st, pf)))
      return rc;
  } else if (slice_beta) {
    if ((rc = oz_slice_rows(beta, npw, np, npw, 0, bs, &A1, st, pf))) return rc;
    if ((rc = oz_slice_cols(beta, npw, np, npw, r4 ? 4 : 0, bs + oz_operand_bytes(np, npw), &A2, st,
                            pf)))
      return rc;
  } else {
    A1 = oz_carve(bs, np, npw);
    A2 = r4 ? oz_carve(bs + oz_operand_bytes(np, npw), 2 * npw, (np + 1) / 2)
            : oz_carve(bs + oz_operand_bytes(np, npw), npw, np);
  }
  char* w = static_cast<char*>(work);
  char* wb1 = w;
  char* part = wb1 + oz_operand_bytes(2 * nb, npw);
  char* wb2 = part + oz_partial_bytes(np, nb, npw);
  double* P = reinterpret_cast<double*>(wb2 + oz_operand_bytes(2 * nb, np));
  P = reinterpret_cast<double*>(((uintptr_t)P + 255) & ~(uintptr_t)255);
  double* Q = reinterpret_cast<double*>(reinterpret_cast<char*>(P) + up256((size_t)np * nb * 16));
  // real_p: only Re P is used, so the real-output product (half the work)
  if ((rc = oz_slice_rows(psi, npw, nb, npw, real_p ? 0 : 1, wb1, &B1, st, pf))) return rc;
  if ((rc = oz_gemm_inner(A1, B1, np, nb, P, nb, part, oz_partial_bytes(np, nb, npw), status, st, pf,
                          real_p)))
    return rc;
  if ((rc = dmul(dmat, P, Q, np, nb, st, pf, real_p))) return rc;
  if (r4) {
    if ((rc = oz_slice_cols(Q, nb, np, nb, 5, wb2, &B2, st, pf))) return rc;
    return oz_launch(A2, B2, 2 * npw, nb, reinterpret_cast<double2*>(hpsi), npw, 0, 1, 0, 1, 2,
                     status, st, pf);
  }
  if ((rc = oz_slice_cols(Q, nb, np, nb, 2, wb2, &B2, st, pf))) return rc;
  return oz_gemm_outer(A2, B2, npw, nb, hpsi, npw, 0, 1, status, st, pf);
}

}  // namespace qe
