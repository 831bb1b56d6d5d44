// tdm_alg2.cu -- Algorithm 2 (Section 3.1): selected components of every
// solution of the series as dense products, x_k = G_k^T F for k in a set of
// P components, all right-hand sides at once:
//
//     X[P][N] = G^T[P][n] F[n][N],     G_k = A^{-1} e_k (eq. green_v, Lemma 2).
//
// The product runs on the 5th-generation tensor cores (tcgen05.mma, kind::tf32)
// with binary32 accumulation in tensor memory, in three TF32 products:
// G^T = Gh + Gl and F = Fh + Fl split into a TF32 head (10 significand bits)
// and the binary32 remainder, X ~ Gh Fh + Gl Fh + Gh Fl (Gl Fl is below the
// product's rounding).
//
// Structure (one CTA per 128 columns of F and one slice of 1024 rows of K = n):
// the CTA computes D^T = F^T G for its 128 columns and all P <= 512 components,
// so its accumulator is 128 TMEM lanes (columns of F) x P TMEM columns.
//   warp 0       allocates the tensor memory; one lane issues the TMA loads of
//                every stage (the F tile [16 rows][128 columns] as stored, and
//                G's head and tail, pre-split by k_alg2_split into the MMA's
//                K-major core-matrix layout);
//   warps 1-4    split each F tile into head and tail and write them in the
//                same K-major layout (the transposition the MMA needs: F's
//                columns are contiguous, the MMA wants K contiguous); after the
//                last stage they read the accumulator out of tensor memory;
//   warp 5       one lane issues the MMAs of a stage once it is converted and
//                commits them to the stage's "empty" barrier.
// Every CTA writes its binary32 partial product of 1024 terms; k_alg2_reduce
// adds the partials of the K slices in binary32 pairs.  Keeping each binary32
// accumulation to 1024 terms bounds the rounding of a product whose terms
// cancel heavily (|x_k| << sum |G_k(i) F_i| for an ill-conditioned A).
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// "core matrices" of 8 rows x 16 bytes (4 binary32), rows 16 bytes apart;
// the next 8 rows 128 bytes further (the descriptor's stride offset); the next
// 4 elements of K one whole row block further (its leading offset).
// Every wait on an mbarrier is bounded; a wait that gives up records device
// error 1, and the CTA skips the rest of its work, waits (bounded) for its own
// issued MMAs and frees the tensor memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "tdm_internal.cuh"
#include "tdm_tma.cuh"

namespace {

constexpr int kBN = 128;       // columns of F per CTA (the MMA's M)
constexpr int kBK = 16;        // rows of K per stage
constexpr int kKS = 1024;      // rows of K per CTA (one binary32 partial)
constexpr int kPmax = 512;     // components per launch (tensor-memory columns)
constexpr int kStages = 2;
constexpr int kThreads = 192;  // warp 0 TMA + TMEM, warps 1-4 convert + epilogue, warp 5 MMA

// shared-memory layout of one stage (bytes)
constexpr uint32_t kBhalf = 256 * kBK * 4;          // one half (256 components) of G's head or tail: 16 KB
constexpr uint32_t kSzB = 2 * kBhalf;               // all 512 components: 32 KB
constexpr uint32_t kSzA = kBN * kBK * 4;            // F's head or tail: 8 KB
constexpr uint32_t kSzF = kBK * kBN * 4;            // F tile as loaded: 8 KB
constexpr uint32_t kOffGh = 0, kOffGl = kSzB, kOffFh = 2 * kSzB, kOffFl = 2 * kSzB + kSzA,
                   kOffF = 2 * kSzB + 2 * kSzA, kStage = 2 * kSzB + 2 * kSzA + kSzF;
constexpr uint32_t kSmemBars = kStages * kStage;    // mbarriers after the stages
constexpr uint32_t kSmemBytes = kSmemBars + 128;

// ---- PTX helpers ---------------------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bounded wait for phase `parity`; false (and device error 1) after ~1 s
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(100000u)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) {
      if (err) atomicExch(err, kDevErrTmaTimeout);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_1d(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance of
// the next 4 elements of K, sbo = byte distance of the next 8 rows.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // fixed constant 0b001 at bits 46-48
  return d;                 // base offset 0, relative leading offset, no swizzle
}
// Instruction descriptor of kind::tf32: D binary32, A and B TF32, both K-major,
// M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4)                      // D format: F32
         | (2u << 7) | (2u << 10)       // A, B format: TF32
         | ((uint32_t)(n >> 3) << 17)   // N / 8
         | ((uint32_t)(128 >> 4) << 24);   // M / 16
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"((int)accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// TF32 head of a binary32 value (significand cut to 10 bits)
__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// ---- G^T head and tail in the MMA layout ---------------------------------------
// Gs[slice][part][stage-in-slice][half][kc][row][4] with part 0 = head, 1 = tail:
// for every stage of kBK rows of K, the 512 components as two blocks of 256 rows,
// each [kBK/4 groups of K][256 rows][4 consecutive K] -- exactly a stage's
// shared-memory image, loaded by one bulk copy.  Components >= P and rows
// >= n are zero.
__global__ void k_alg2_split(const double* __restrict__ G, int64_t ldG, int P, int64_t n, int64_t Kp,
                             float* __restrict__ Gs) {
  const int64_t total = (int64_t)kPmax * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % kPmax);
    const int64_t k = e / kPmax;
    const double g = (p < P && k < n) ? G[k * ldG + p] : 0.0;
    const float h = tf32_head((float)g);
    const float l = (float)(g - (double)h);
    const int64_t st = k / kBK;            // stage (global)
    const int kk = (int)(k % kBK);
    const int half = p / 256, row = p % 256;
    const size_t within = ((size_t)half * (kBK / 4) + kk / 4) * 256 * 4 + (size_t)row * 4 + (kk & 3);
    const size_t base = (size_t)st * 2 * (kSzB / 4);   // head and tail of every stage
    Gs[base + within] = h;
    Gs[base + kSzB / 4 + within] = l;
  }
}

struct Alg2Args {
  const float* Gs;     // split G^T (k_alg2_split)
  float* part;         // [slices][kPmax][Npad] binary32 partials
  int64_t Npad;
  int64_t N, Kp;
  int P;
  int* err;
};

__global__ void __launch_bounds__(kThreads, 1) k_alg2_tc(const __grid_constant__ CUtensorMap tmF, const Alg2Args a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col0 = blockIdx.x * kBN;                       // first column of F
  const int slice = blockIdx.y;                            // K slice
  const int64_t k0 = (int64_t)slice * kKS;
  const int64_t k1 = k0 + kKS < a.Kp ? k0 + kKS : a.Kp;
  const int nst = (int)((k1 - k0) / kBK);                  // stages of this CTA
  const uint32_t sbase = saddr(sm);
  const uint32_t bar_full = sbase + kSmemBars;             // [kStages] TMA done
  const uint32_t bar_conv = bar_full + 8 * kStages;        // [kStages] head / tail of F written
  const uint32_t bar_empty = bar_conv + 8 * kStages;       // [kStages] the stage's MMAs done
  const uint32_t bar_done = bar_empty + 8 * kStages;       // every MMA done

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_conv + 8 * s, 4);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_s = 0;
  }
  if (warp == 0) {   // the accumulator: 128 lanes x 512 columns of binary32
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base_s)),
                 "r"(kPmax)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  bool ok = true;

  if (warp == 0) {
    // ---- TMA producer ------------------------------------------------------------
    if (lane == 0) {
      for (int i = 0; i < nst && ok; i++) {
        const int s = i % kStages;
        const uint32_t par = ((i / kStages) & 1) ^ 1;
        if (!mbar_wait(bar_empty + 8 * s, par, a.err)) { ok = false; break; }
        const uint32_t st = sbase + s * kStage;
        mbar_expect_tx(bar_full + 8 * s, 2 * kSzB + kSzF);
        const int64_t gst = k0 / kBK + i;   // global stage of G
        tma_1d(st + kOffGh, a.Gs + (size_t)gst * 2 * (kSzB / 4), 2 * kSzB, bar_full + 8 * s);   // head and tail
        tma_2d(st + kOffF, &tmF, col0, (int)(k0 + (int64_t)i * kBK), bar_full + 8 * s);
      }
      if (!ok) atomicExch(&abort_s, 1);
    }
  } else if (warp == 5) {
    // ---- MMA issuer --------------------------------------------------------------
    if (lane == 0) {
      const uint32_t id = idesc_tf32(256);
      for (int i = 0; i < nst && ok; i++) {
        const int s = i % kStages;
        if (!mbar_wait(bar_conv + 8 * s, (i / kStages) & 1, a.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t st = sbase + s * kStage;
#pragma unroll
        for (int kk = 0; kk < kBK / 8; kk++) {   // K = 8 per MMA: two groups of 4
#pragma unroll
          for (int h = 0; h < 2; h++) {          // components 0-255, 256-511
            const uint64_t fh = sdesc(st + kOffFh + kk * 2 * (kBN * 16), kBN * 16, 128);
            const uint64_t fl = sdesc(st + kOffFl + kk * 2 * (kBN * 16), kBN * 16, 128);
            const uint64_t gh = sdesc(st + kOffGh + h * kBhalf + kk * 2 * (256 * 16), 256 * 16, 128);
            const uint64_t gl = sdesc(st + kOffGl + h * kBhalf + kk * 2 * (256 * 16), 256 * 16, 128);
            const uint32_t d = tmem + h * 256;
            mma_tf32(d, fh, gh, id, i > 0 || kk > 0);
            mma_tf32(d, fh, gl, id, true);
            mma_tf32(d, fl, gh, id, true);
          }
        }
        mma_commit(bar_empty + 8 * s);   // frees the stage once these MMAs have read it
      }
      mma_commit(bar_done);              // every MMA issued so far (also on the error path)
      if (!ok) atomicExch(&abort_s, 1);
    }
  } else {
    // ---- F head and tail, then the epilogue (warps 1-4) ----------------------------
    const int m = threadIdx.x - 32;   // column of the tile (TMEM lane)
    for (int i = 0; i < nst && ok; i++) {
      const int s = i % kStages;
      if (!mbar_wait(bar_full + 8 * s, (i / kStages) & 1, a.err)) { ok = false; break; }
      const float* Ft = reinterpret_cast<const float*>(sm + s * kStage + kOffF);   // [kBK][kBN]
      float4* Fh = reinterpret_cast<float4*>(sm + s * kStage + kOffFh);           // [kBK/4][kBN] of 4
      float4* Fl = reinterpret_cast<float4*>(sm + s * kStage + kOffFl);
#pragma unroll
      for (int kc = 0; kc < kBK / 4; kc++) {
        float4 v;
        v.x = Ft[(4 * kc + 0) * kBN + m];
        v.y = Ft[(4 * kc + 1) * kBN + m];
        v.z = Ft[(4 * kc + 2) * kBN + m];
        v.w = Ft[(4 * kc + 3) * kBN + m];
        const float4 h = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
        Fh[kc * kBN + m] = h;
        Fl[kc * kBN + m] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
      }
      fence_proxy_async();   // the generic writes, visible to the tensor cores
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_conv + 8 * s);
    }
    // the accumulator, once every MMA has completed
    const bool done = mbar_wait(bar_done, 0, a.err);
    tc_fence_after();
    if (ok && done && !abort_s) {
      const int q = warp & 3;                               // lanes 32q .. 32q+31 of tensor memory
      const int64_t col = (int64_t)col0 + 32 * q + lane;   // column of F
      float* out = a.part + (size_t)slice * kPmax * a.Npad + col;
      for (int c0 = 0; c0 < kPmax; c0 += 32) {
        if (c0 >= a.P) break;
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (col < a.N) {
#pragma unroll
          for (int j = 0; j < 32; j++)
            if (c0 + j < a.P) out[(size_t)(c0 + j) * a.Npad] = __uint_as_float(r[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPmax) : "memory");
  }
}

// X[p][c] = sum over the K slices of the partials, in binary32 pairs (TwoSum),
// rounded once to binary32
__global__ void k_alg2_reduce(const float* __restrict__ part, int slices, int P, int64_t N, int64_t Npad,
                              float* __restrict__ X, int64_t ldX) {
  const int64_t total = (int64_t)P * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / N);
    const int64_t c = e % N;
    float hi = 0.f, lo = 0.f;
    for (int s = 0; s < slices; s++) {
      const float v = part[((size_t)s * kPmax + p) * Npad + c];
      const float t = hi + v;
      const float bb = t - hi;
      lo += (hi - (t - bb)) + (v - bb);
      hi = t;
    }
    X[p * ldX + c] = hi + lo;
  }
}

bool encode_f(CUtensorMap* out, const float* F, int64_t ldF, int64_t N, int64_t n) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      (void)cudaGetLastError();
  });
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ldF * 4};
  cuuint32_t box[2] = {kBN, kBK};
  cuuint32_t estr[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(F), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

extern "C" size_t tdm_algorithm2_workspace(int64_t P, int64_t n, int64_t N) {
  if (P < 0 || n < 1 || N < 0) return 0;
  const int64_t Kp = round_up(n, kBK), slices = (Kp + kKS - 1) / kKS, Npad = round_up(N > 0 ? N : 1, kBN);
  const int64_t blocks = (P + kPmax - 1) / kPmax;
  (void)blocks;
  return (size_t)(2 * kPmax * Kp) * 4 + (size_t)(slices * kPmax * Npad) * 4 + 256;
}

extern "C" tdm_status tdm_algorithm2(const double* G, int64_t ldG, int64_t P, int64_t n, const float* F, int64_t ldF,
                                     int64_t N, float* X, int64_t ldX, void* work, size_t work_bytes, void* stream) {
  if (P < 0 || n < 1 || N < 0) return TDM_ERR_INVALID_ARG;
  if (P == 0 || N == 0) return TDM_OK;
  if (!G || !F || !X || !work || ldG < P || ldF < N || ldX < N) return TDM_ERR_INVALID_ARG;
  if (!tdm_aligned(F, 16) || (ldF % 4) || !tdm_aligned(work, 256) || !tdm_aligned(G, 8)) return TDM_ERR_INVALID_ARG;
  if (n > (int64_t(1) << 30) || N > (int64_t(1) << 30)) return TDM_ERR_INVALID_ARG;
  if (work_bytes < tdm_algorithm2_workspace(P < kPmax ? P : kPmax, n, N)) return TDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  const int64_t Kp = round_up(n, kBK), slices = (Kp + kKS - 1) / kKS, Npad = round_up(N, kBN);
  float* Gs = static_cast<float*>(work);
  float* part = Gs + 2 * kPmax * Kp;
  int* err = nullptr;   // device errors go to the first word past the partials
  err = reinterpret_cast<int*>(part + slices * kPmax * Npad);
  CUtensorMap tmF;
  memset(&tmF, 0, sizeof(tmF));
  if (!encode_f(&tmF, F, ldF, N, n)) return TDM_ERR_NOT_IMPLEMENTED;
  static bool attr_set = false;
  if (!attr_set) {
    TDM_CUDA_TRY(cudaFuncSetAttribute(k_alg2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
    attr_set = true;
  }
  TDM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  for (int64_t p0 = 0; p0 < P; p0 += kPmax) {   // blocks of 512 components
    const int Pb = (int)(P - p0 < kPmax ? P - p0 : kPmax);
    const int64_t total = (int64_t)kPmax * Kp;
    k_alg2_split<<<(int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192), 256, 0, s>>>(G + p0, ldG, Pb, n, Kp, Gs);
    Alg2Args a;
    a.Gs = Gs; a.part = part; a.Npad = Npad; a.N = N; a.Kp = Kp; a.P = Pb; a.err = err;
    const dim3 grid((unsigned)(Npad / kBN), (unsigned)slices);
    k_alg2_tc<<<grid, kThreads, kSmemBytes, s>>>(tmF, a);
    const int64_t tot2 = (int64_t)Pb * N;
    k_alg2_reduce<<<(int)((tot2 + 255) / 256 < 8192 ? (tot2 + 255) / 256 : 8192), 256, 0, s>>>(
        part, (int)slices, Pb, N, Npad, X + p0 * ldX, ldX);
    TDM_CUDA_TRY(cudaGetLastError());
  }
  return TDM_OK;
}

// The device error word of the last call (0 = none, 1 = a bounded wait gave up);
// synchronizes the stream.
extern "C" tdm_status tdm_algorithm2_status(const void* work, int64_t P, int64_t n, int64_t N, void* stream,
                                            int* device_error) {
  if (!work || !device_error) return TDM_ERR_INVALID_ARG;
  const int64_t Kp = round_up(n, kBK), slices = (Kp + kKS - 1) / kKS, Npad = round_up(N > 0 ? N : 1, kBN);
  const float* part = static_cast<const float*>(work) + 2 * kPmax * Kp;
  const int* err = reinterpret_cast<const int*>(part + slices * kPmax * Npad);
  (void)P;
  cudaStream_t s = (cudaStream_t)stream;
  TDM_CUDA_TRY(cudaMemcpyAsync(device_error, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TDM_CUDA_TRY(cudaStreamSynchronize(s));
  return TDM_OK;
}
