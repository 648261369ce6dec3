// The learned radiance cache: a 3 x 64 MLP R(x, d) over a frequency encoding
// of position and direction, trained online on the tracer's own path vertices
// and used to end paths after one or two collisions (the cached estimator).
//
// Tensor-core design (sm_100 family, tcgen05).  A block of 128 threads owns a
// tile of 128 records, thread t row t.  Every matrix product of the network is
// D[128 x N] (+)= A[128 x K] B[N x K]^T with BF16 operands in shared memory and
// the FP32 accumulator D in tensor memory (TMEM, row i = lane i):
//   * operands use the canonical no-swizzle K-major layout: 8 x 16-byte core
//     matrices (8 rows x 8 bf16), cores adjacent in K 128 bytes apart (leading
//     byte offset), 8-row groups `sbo` bytes apart (stride byte offset);
//   * one thread issues K / 16 tcgen05.mma instructions (M = 128, N = 64 or
//     128, K = 16 each) and a tcgen05.commit onto an mbarrier; the block waits
//     on the barrier (bounded), then every warp reads its 32 TMEM lanes with
//     tcgen05.ld for the epilogue on the CUDA cores (bias, ReLU, rounding to
//     bf16 into the next operand, output layer, loss).
// Training runs forward and backward in the same kernel.  Weight gradients
// dW = dZ^T H use the transposed activations as operands (written transposed
// in the epilogues) and accumulate in TMEM across all tiles of a block; only
// the block's final sums go to global memory.  Bias gradients stay FP32:
// reduced across each warp with a recursive-halving butterfly.
#include <cuda_bf16.h>

#include "walk_tet.cuh"

namespace tv {
namespace rc {

constexpr int WID = 64, ENC = 128, PFREQ = 12, DFREQ = 4;
constexpr int O_W1 = 0, O_B1 = O_W1 + WID * ENC, O_W2 = O_B1 + WID, O_B2 = O_W2 + WID * WID, O_W3 = O_B2 + WID,
              O_B3 = O_W3 + WID * WID, O_W4 = O_B3 + WID, O_B4 = O_W4 + WID, NPARAM = O_B4 + 1;
static_assert(NPARAM == RC_NUM_PARAMS, "parameter layout");
static_assert(O_W1 % 4 == 0 && O_W2 % 4 == 0 && O_W3 % 4 == 0, "weight blocks start on 16-byte boundaries");
constexpr int MT = 128;                      // rows per tile (MMA M) = threads per block
constexpr int SBO64 = 1024, SBO128 = 2048;   // 8-row-group stride of a K = 64 / K = 128 operand
constexpr long long WAIT_LIMIT = 1ll << 22;  // mbarrier polls before a wait gives up

__device__ unsigned long long g_timeouts = 0;

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the barrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_test(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, leading byte offset 128 (K-adjacent cores).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// D (+)= A B^T over K = 16 * ksteps: A (128 rows) and B (N rows) canonical K-major.
__device__ __forceinline__ void gemm(uint32_t d, const void* A, uint32_t a_sbo, const void* B, uint32_t b_sbo,
                                     int ksteps, uint32_t idesc, bool accumulate) {
  const uint32_t a = smem_addr(A), b = smem_addr(B);
  for (int s = 0; s < ksteps; ++s)
    mma(d, sdesc(a + 256u * s, a_sbo), sdesc(b + 256u * s, b_sbo), idesc, (accumulate || s > 0) ? 1u : 0u);
}

#define TV_TMEM_LD16(taddr, r)                                                                                   \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, " \
               "[%16];"                                                                                          \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),         \
                 "=r"(r[15])                                                                                     \
               : "r"(taddr))

// 4 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ float4 tmem_ld4(uint32_t taddr) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  return make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
}

// dst[0..64) += the 64 FP32 columns of this thread's TMEM lane at taddr, with
// 16-byte atomics (dst 16-byte aligned).  The block starts at its own group of
// four columns, so that blocks finishing together spread their atomics over 16
// address groups instead of all adding into the same addresses at once.
__device__ __forceinline__ void tmem_add_row64(uint32_t taddr, float* dst) {
  const int rot = (int)(blockIdx.x & 15u);
#pragma unroll 4
  for (int k = 0; k < 16; ++k) {
    const int c = ((k + rot) & 15) * 4;
    atomicAdd(reinterpret_cast<float4*>(dst + c), tmem_ld4(taddr + (uint32_t)c));
  }
}

// 64 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r0[16], r1[16], r2[16], r3[16];
  TV_TMEM_LD16(taddr, r0);
  TV_TMEM_LD16(taddr + 16, r1);
  TV_TMEM_LD16(taddr + 32, r2);
  TV_TMEM_LD16(taddr + 48, r3);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] = __uint_as_float(r0[i]);
    v[16 + i] = __uint_as_float(r1[i]);
    v[32 + i] = __uint_as_float(r2[i]);
    v[48 + i] = __uint_as_float(r3[i]);
  }
}

// ---------------------------------------------------------------------------
// operand layout helpers
// ---------------------------------------------------------------------------
// byte offset of element (r, k) of a canonical K-major operand
__device__ __forceinline__ uint32_t cofs(int r, int k, uint32_t sbo) {
  return (uint32_t)(r >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);     // a in the low half (lower address)
  return *reinterpret_cast<const uint32_t*>(&h);
}

// 8 consecutive K elements (k multiple of 8) of row r, rounded to bf16
__device__ __forceinline__ void put8(uint8_t* base, int r, int k, uint32_t sbo, const float* v) {
  *reinterpret_cast<uint4*>(base + cofs(r, k, sbo)) =
      make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}

__device__ __forceinline__ void put1(uint8_t* base, int r, int k, uint32_t sbo, __nv_bfloat16 v) {
  *reinterpret_cast<__nv_bfloat16*>(base + cofs(r, k, sbo)) = v;
}

// a rows x K fp32 matrix M[r][k] (or its transpose, M[k][r], when T) into a
// canonical bf16 operand; all threads of the block
template <bool T>
__device__ void load_matrix(uint8_t* dst, const float* M, int rows, int K, uint32_t sbo) {
  const int chunks = rows * K / 8;
  for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
    const int r = i / (K / 8), k = (i % (K / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = T ? M[(k + j) * rows + r] : M[r * K + k + j];
    put8(dst, r, k, sbo, v);
  }
}

// ---------------------------------------------------------------------------
// the frequency encoding, 8 features at a time: chunk c covers features 8c..8c+7
// ---------------------------------------------------------------------------
// sin(pi u) and cos(pi u): with k = rint(u), u - k is exact and sin(pi u) =
// (-1)^k sin(pi (u - k)), cos(pi u) = (-1)^k cos(pi (u - k)); the angle is in
// [-pi/2, pi/2], where the hardware approximations' absolute error is below
// 2^-21 -- far below the bf16 rounding the features go through (2^-9 relative).
__device__ __forceinline__ void sincospi_enc(float u, float* s, float* c) {
  const float k = rintf(u);
  const float th = (u - k) * 3.14159265358979f;
  const uint32_t odd = ((uint32_t)__float2int_rn(k) & 1u) << 31;
  *s = __uint_as_float(__float_as_uint(__sinf(th)) ^ odd);
  *c = __uint_as_float(__float_as_uint(__cosf(th)) ^ odd);
}

template <class Sink>
__device__ __forceinline__ void encode(const float x[3], const float d[3], Sink&& sink) {
#pragma unroll
  for (int c = 0; c < ENC / 8; ++c) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = 4 * c + j;                  // feature pair (2p, 2p + 1)
      float a, b;
      if (p == 0) { a = x[0]; b = x[1]; }
      else if (p == 1) { a = x[2]; b = d[0]; }
      else if (p == 2) { a = d[1]; b = d[2]; }
      else if (p < 3 + 3 * PFREQ) {
        const int q = p - 3;                    // sin and cos of 2^l pi x_a
        sincospi_enc(x[q / PFREQ] * (float)(1 << (q % PFREQ)), &a, &b);
      } else if (p < 3 + 3 * PFREQ + 3 * DFREQ) {
        const int q = p - 3 - 3 * PFREQ;        // sin and cos of 2^l pi d_a
        sincospi_enc(d[q / DFREQ] * (float)(1 << (q % DFREQ)), &a, &b);
      } else {
        a = b = 0.f;
      }
      v[2 * j] = a;
      v[2 * j + 1] = b;
    }
    sink(c, v);
  }
}

// Warp sums of 64 per-lane columns: afterwards lane l holds the sums of columns
// 2l and 2l + 1 (recursive halving: each level swaps the half a lane gives away).
__device__ __forceinline__ float2 warp_colsum64(float (&v)[64]) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int h = 64, off = 16; off >= 1; h >>= 1, off >>= 1) {
    const bool upper = (lane & (unsigned)off) != 0;
#pragma unroll
    for (int i = 0; i < h / 2; ++i) {
      const float keep = upper ? v[h / 2 + i] : v[i];
      const float give = upper ? v[i] : v[h / 2 + i];
      v[i] = keep + __shfl_xor_sync(~0u, give, off);
    }
  }
  return make_float2(v[0], v[1]);
}

// Block-wide handshake before the tensor cores read operands written by threads.
__device__ __forceinline__ void operands_ready() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_before();
  __syncthreads();
  tc_after();
}

// Wait for the MMAs committed to `bar` (all threads); false for the whole block
// if any thread's wait ran out.
__device__ __forceinline__ bool mma_done(uint64_t* bar, uint32_t& phase) {
  const bool ok = mbar_wait(bar, phase);
  phase ^= 1u;
  const bool all = __syncthreads_and(ok) != 0;
  tc_after();
  return all;
}

// ---------------------------------------------------------------------------
// inference: R(x, d) per record; COMPOSE writes L + beta * max(R, 0) into the
// record's L slot instead (the cached estimator)
//
// One block per SM holds the weights once and runs IG groups of 128 threads,
// each with its own 128-row tile, operand buffer, TMEM accumulator (64 columns)
// and mbarrier, so that one group's encoding and epilogues run while other
// groups' MMAs are in flight.  Group g is warps 4g..4g+3: warp w reads TMEM
// lanes 32 (w mod 4).. as tcgen05.ld requires, and the group synchronises on
// its own named barrier.
// ---------------------------------------------------------------------------
constexpr int IG = 6;

struct InferSmem {
  alignas(128) uint8_t W1[WID * ENC * 2];
  alignas(128) uint8_t W2[WID * WID * 2];
  alignas(128) uint8_t W3[WID * WID * 2];
  alignas(128) uint8_t X[IG][MT * ENC * 2];
  float b1[WID], b2[WID], b3[WID], w4[WID];
  float b4;
  alignas(8) uint64_t bar[IG];
  uint32_t tmem;
};

// named barrier of one group (id 1 + g, 128 threads); returns the AND / OR of v over the group
__device__ __forceinline__ bool group_and(int id, bool v) {
  uint32_t r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.and.pred q, %2, 128, p;\n"
               " selp.u32 %0, 1, 0, q;\n}"
               : "=r"(r)
               : "r"((uint32_t)v), "r"(id)
               : "memory");
  return r != 0;
}
__device__ __forceinline__ bool group_or(int id, bool v) {
  uint32_t r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.or.pred q, %2, 128, p;\n"
               " selp.u32 %0, 1, 0, q;\n}"
               : "=r"(r)
               : "r"((uint32_t)v), "r"(id)
               : "memory");
  return r != 0;
}
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("barrier.cta.sync %0, 128;" ::"r"(id) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r0[16], r1[16];
  TV_TMEM_LD16(taddr, r0);
  TV_TMEM_LD16(taddr + 16, r1);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] = __uint_as_float(r0[i]);
    v[16 + i] = __uint_as_float(r1[i]);
  }
}

template <bool COMPOSE>
__global__ void __launch_bounds__(IG * MT, 1) k_mlp_infer(const float* __restrict__ P, float* rec, long long n,
                                                          float* __restrict__ y) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  InferSmem& S = *reinterpret_cast<InferSmem*>(smem_raw);
  const int g = threadIdx.x / MT, t = threadIdx.x % MT, warp = threadIdx.x >> 5;
  const int bid = 1 + g;                          // the group's named barrier
  if (warp == 0) tmem_alloc(&S.tmem, 512);
  if (threadIdx.x < IG) mbar_init(&S.bar[threadIdx.x]);
  load_matrix<false>(S.W1, P + O_W1, WID, ENC, SBO128);
  load_matrix<false>(S.W2, P + O_W2, WID, WID, SBO64);
  load_matrix<false>(S.W3, P + O_W3, WID, WID, SBO64);
  if (threadIdx.x < WID) {
    const int c = threadIdx.x;
    S.b1[c] = P[O_B1 + c]; S.b2[c] = P[O_B2 + c]; S.b3[c] = P[O_B3 + c]; S.w4[c] = P[O_W4 + c];
  }
  if (threadIdx.x == 0) S.b4 = P[O_B4];
  tc_before();
  __syncthreads();
  tc_after();
  uint8_t* X = S.X[g];
  uint64_t* bar = &S.bar[g];
  const uint32_t D = S.tmem + (uint32_t)(g * 64), Drow = D + ((uint32_t)((warp & 3) * 32) << 16);
  uint32_t phase = 0;
  bool ok = true;
  const long long ntiles = (n + MT - 1) / MT;
  for (long long tile = (long long)blockIdx.x * IG + g; tile < ntiles; tile += (long long)gridDim.x * IG) {
    const long long row = tile * MT + t;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (row < n) {
      r0 = reinterpret_cast<const float4*>(rec)[2 * row];
      r1 = reinterpret_cast<const float4*>(rec)[2 * row + 1];
    }
    // a cached frame's tile without a single query (every path ended before its
    // cache collision) needs no network: its records already hold their estimates
    if (COMPOSE && !group_or(bid, r0.w > 0.f)) continue;
    const float x[3] = {r0.x, r0.y, r0.z}, d[3] = {r1.x, r1.y, r1.z};
    encode(x, d, [&](int c, const float* v) { put8(X, t, 8 * c, SBO128, v); });
    float out = S.b4;
    // three hidden layers; the first reads the 128-wide encoding
#pragma unroll 1
    for (int layer = 0; layer < 3; ++layer) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_before();
      group_sync(bid);
      tc_after();
      if (t == 0) {
        if (layer == 0) gemm(D, X, SBO128, S.W1, SBO128, ENC / 16, idesc_bf16(MT, WID), false);
        else gemm(D, X, SBO64, layer == 1 ? S.W2 : S.W3, SBO64, WID / 16, idesc_bf16(MT, WID), false);
        mma_commit(bar);
      }
      const bool mine = mbar_wait(bar, phase);
      phase ^= 1u;
      ok = group_and(bid, mine) && ok;
      tc_after();
      if (!ok) break;
      // the epilogue in two halves of 32 columns (fewer live registers)
#pragma unroll
      for (int hlf = 0; hlf < 2; ++hlf) {
        float v[32];
        tmem_ld32(Drow + 32u * hlf, v);
        if (layer < 2) {
          const float* b = (layer == 0 ? S.b1 : S.b2) + 32 * hlf;
#pragma unroll
          for (int c = 0; c < 32; c += 8) {
            float h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = fmaxf(v[c + j] + b[c + j], 0.f);
            put8(X, t, 32 * hlf + c, SBO64, h);
          }
        } else {
#pragma unroll
          for (int c = 0; c < 32; ++c) out += S.w4[32 * hlf + c] * fmaxf(v[c] + S.b3[32 * hlf + c], 0.f);
        }
      }
    }
    if (!ok) {
      if (row < n) {
        if (COMPOSE) rec[8 * row + 7] = __int_as_float(0x7FC00000);
        else y[row] = __int_as_float(0x7FC00000);
      }
      break;
    }
    if (row < n) {
      if (COMPOSE) rec[8 * row + 7] = r1.w + r0.w * fmaxf(out, 0.f);
      else y[row] = out;
    }
    // the next tile's operands overwrite X: every thread of the group is past its last read
    // of it (the layer-3 MMA has completed; the epilogue reads TMEM only)
  }
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    tmem_dealloc(S.tmem, 512);
  }
  if (!ok && t == 0) atomicAdd(&g_timeouts, 1ull);
}

// ---------------------------------------------------------------------------
// training: forward, L2 loss and backward over tiles of samples
// ---------------------------------------------------------------------------
struct GradSmem {
  alignas(128) uint8_t W1[WID * ENC * 2];     // B of layer 1       [64 out][128 in]
  alignas(128) uint8_t W2[WID * WID * 2];     // B of layer 2       [64 out][64 in]
  alignas(128) uint8_t W3[WID * WID * 2];
  alignas(128) uint8_t W2T[WID * WID * 2];    // B of dH1 = dZ2 W2  [64 in][64 out]
  alignas(128) uint8_t W3T[WID * WID * 2];
  alignas(128) uint8_t X[MT * ENC * 2];       // A of the forward layers: e, then h1, h2
  alignas(128) uint8_t ET[ENC * MT * 2];      // e^T  [128 feature][128 row]  (B of dW1)
  alignas(128) uint8_t H1T[WID * MT * 2];     // h1^T [64][128]               (B of dW2)
  alignas(128) uint8_t H2T[WID * MT * 2];     // h2^T                         (B of dW3)
  alignas(128) uint8_t DZ[MT * WID * 2];      // dZ   [128 row][64]           (A of dH)
  alignas(128) uint8_t DZT[MT * MT * 2];      // dZ^T [64 (+64 zero) out][128 row] (A of dW)
  float b1[WID], b2[WID], b3[WID], w4[WID];
  float gb1[WID], gb2[WID], gb3[WID], gw4[WID];
  float b4, gb4, loss, count;
  alignas(8) uint64_t bar;
  uint32_t tmem;
};

// TMEM columns of the training kernel
constexpr uint32_t T_F = 0, T_X = 64, T_W1 = 128, T_W2 = 256, T_W3 = 320, T_COLS = 512;

__global__ void __launch_bounds__(MT, 1) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ smp,
                                                    long long n, float* __restrict__ grad,
                                                    float* __restrict__ loss_out) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (warp == 0) tmem_alloc(&S.tmem, T_COLS);
  if (t == 0) {
    mbar_init(&S.bar);
    S.b4 = P[O_B4];
    S.gb4 = 0.f; S.loss = 0.f; S.count = 0.f;
  }
  load_matrix<false>(S.W1, P + O_W1, WID, ENC, SBO128);
  load_matrix<false>(S.W2, P + O_W2, WID, WID, SBO64);
  load_matrix<false>(S.W3, P + O_W3, WID, WID, SBO64);
  load_matrix<true>(S.W2T, P + O_W2, WID, WID, SBO64);
  load_matrix<true>(S.W3T, P + O_W3, WID, WID, SBO64);
  if (t < WID) {
    S.b1[t] = P[O_B1 + t]; S.b2[t] = P[O_B2 + t]; S.b3[t] = P[O_B3 + t]; S.w4[t] = P[O_W4 + t];
    S.gb1[t] = 0.f; S.gb2[t] = 0.f; S.gb3[t] = 0.f; S.gw4[t] = 0.f;
  }
  // rows 64..127 of dZ^T stay zero: the weight-gradient MMA runs at M = 128
  for (int i = t; i < MT * MT * 2 / 16; i += MT) reinterpret_cast<uint4*>(S.DZT)[i] = make_uint4(0, 0, 0, 0);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t base = S.tmem, lanes = (uint32_t)(warp * 32) << 16;
  const uint32_t DF = base + T_F, DX = base + T_X;
  uint32_t phase = 0;
  bool ok = true, any = false;
  float my_loss = 0.f, my_count = 0.f, my_gb4 = 0.f;
  const long long ntiles = (n + MT - 1) / MT;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long row = tile * MT + t;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (row < n) {
      r0 = reinterpret_cast<const float4*>(smp)[2 * row];
      r1 = reinterpret_cast<const float4*>(smp)[2 * row + 1];
    }
    const float x[3] = {r0.x, r0.y, r0.z}, d[3] = {r1.x, r1.y, r1.z};
    const float target = r0.w, valid = r1.w;
    encode(x, d, [&](int c, const float* v) {
      put8(S.X, t, 8 * c, SBO128, v);
#pragma unroll
      for (int j = 0; j < 8; ++j) put1(S.ET, 8 * c + j, t, SBO128, __float2bfloat16_rn(v[j]));
    });
    float v[64];
    uint32_t mask[3][2];                                 // ReLU masks of z1, z2, z3 (bit c: z_c > 0)
    // ---- forward ----
#pragma unroll 1
    for (int layer = 0; layer < 3; ++layer) {
      operands_ready();
      if (t == 0) {
        if (layer == 0) gemm(DF, S.X, SBO128, S.W1, SBO128, ENC / 16, idesc_bf16(MT, WID), false);
        else gemm(DF, S.X, SBO64, layer == 1 ? S.W2 : S.W3, SBO64, WID / 16, idesc_bf16(MT, WID), false);
        mma_commit(&S.bar);
      }
      ok = mma_done(&S.bar, phase);
      if (!ok) break;
      tmem_ld64(DF + lanes, v);
      const float* b = layer == 0 ? S.b1 : layer == 1 ? S.b2 : S.b3;
      uint32_t m0 = 0, m1 = 0;
#pragma unroll
      for (int c = 0; c < WID; ++c) {
        const float z = v[c] + b[c];
        if (z > 0.f) { if (c < 32) m0 |= 1u << c; else m1 |= 1u << (c - 32); }
        v[c] = fmaxf(z, 0.f);
      }
      mask[layer][0] = m0; mask[layer][1] = m1;
      if (layer < 2) {
        uint8_t* HT = layer == 0 ? S.H1T : S.H2T;
#pragma unroll
        for (int c = 0; c < WID; c += 8) {
          put8(S.X, t, c, SBO64, v + c);
#pragma unroll
          for (int j = 0; j < 8; ++j) put1(HT, c + j, t, SBO128, __float2bfloat16_rn(v[c + j]));
        }
      }
    }
    if (!ok) break;
    any = true;
    // ---- output layer and loss (v = h3) ----
    float out = S.b4;
#pragma unroll
    for (int c = 0; c < WID; ++c) out += S.w4[c] * v[c];
    const float res = out - target;
    const float dy = valid * 2.f * res;
    my_loss += valid * res * res;
    my_count += valid;
    my_gb4 += dy;
    // ---- backward: dZ3 = dy w4 (masked); grad w4 = sum dy h3 ----
    float g[64];
#pragma unroll
    for (int c = 0; c < WID; ++c) g[c] = dy * v[c];
    {
      const float2 s = warp_colsum64(g);
      atomicAdd(&S.gw4[2 * lane], s.x);
      atomicAdd(&S.gw4[2 * lane + 1], s.y);
    }
#pragma unroll 1
    for (int layer = 2; layer >= 0; --layer) {
      // v := dZ of this layer (fp32), from dy (layer 3) or from dH in TMEM
      if (layer == 2) {
#pragma unroll
        for (int c = 0; c < WID; ++c) v[c] = dy * S.w4[c];
      } else {
        tmem_ld64(DX + lanes, v);
      }
      const uint32_t m0 = mask[layer][0], m1 = mask[layer][1];
#pragma unroll
      for (int c = 0; c < WID; ++c) {
        const bool on = c < 32 ? ((m0 >> c) & 1u) : ((m1 >> (c - 32)) & 1u);
        if (!on) v[c] = 0.f;
      }
      // dZ (bf16) as the A operand of dH and, transposed, of dW
#pragma unroll
      for (int c = 0; c < WID; c += 8) {
        if (layer > 0) put8(S.DZ, t, c, SBO64, v + c);
#pragma unroll
        for (int j = 0; j < 8; ++j) put1(S.DZT, c + j, t, SBO128, __float2bfloat16_rn(v[c + j]));
      }
      {
        float* gb = layer == 0 ? S.gb1 : layer == 1 ? S.gb2 : S.gb3;
        const float2 s = warp_colsum64(v);
        atomicAdd(&gb[2 * lane], s.x);
        atomicAdd(&gb[2 * lane + 1], s.y);
      }
      operands_ready();
      if (t == 0) {
        const bool acc = tile != blockIdx.x;             // weight gradients accumulate across tiles
        if (layer == 2) {
          gemm(base + T_W3, S.DZT, SBO128, S.H2T, SBO128, MT / 16, idesc_bf16(MT, WID), acc);
          gemm(DX, S.DZ, SBO64, S.W3T, SBO64, WID / 16, idesc_bf16(MT, WID), false);
        } else if (layer == 1) {
          gemm(base + T_W2, S.DZT, SBO128, S.H1T, SBO128, MT / 16, idesc_bf16(MT, WID), acc);
          gemm(DX, S.DZ, SBO64, S.W2T, SBO64, WID / 16, idesc_bf16(MT, WID), false);
        } else {
          gemm(base + T_W1, S.DZT, SBO128, S.ET, SBO128, MT / 16, idesc_bf16(MT, ENC), acc);
        }
        mma_commit(&S.bar);
      }
      ok = mma_done(&S.bar, phase);
      if (!ok) break;
    }
  }
  // ---- block results to global memory ----
  if (ok && any) {
    // weight gradients: TMEM rows 0..63 (warps 0 and 1) hold dW[out][in]; every row
    // offset below is a multiple of four floats (O_W1, O_W2, O_W3 and the row widths are)
    if (warp < 2) {
      const int o = t;
      tmem_add_row64(base + T_W1 + lanes, grad + O_W1 + o * ENC);
      tmem_add_row64(base + T_W1 + 64 + lanes, grad + O_W1 + o * ENC + 64);
      tmem_add_row64(base + T_W2 + lanes, grad + O_W2 + o * WID);
      tmem_add_row64(base + T_W3 + lanes, grad + O_W3 + o * WID);
    }
    for (int o = 16; o; o >>= 1) {
      my_loss += __shfl_xor_sync(~0u, my_loss, o);
      my_count += __shfl_xor_sync(~0u, my_count, o);
      my_gb4 += __shfl_xor_sync(~0u, my_gb4, o);
    }
    if (lane == 0) {
      atomicAdd(&S.loss, my_loss);
      atomicAdd(&S.count, my_count);
      atomicAdd(&S.gb4, my_gb4);
    }
    __syncthreads();
    if (t < WID) {
      atomicAdd(grad + O_B1 + t, S.gb1[t]);
      atomicAdd(grad + O_B2 + t, S.gb2[t]);
      atomicAdd(grad + O_B3 + t, S.gb3[t]);
      atomicAdd(grad + O_W4 + t, S.gw4[t]);
    }
    if (t == 0) {
      atomicAdd(grad + O_B4, S.gb4);
      atomicAdd(loss_out + 0, S.loss);
      atomicAdd(loss_out + 1, S.count);
    }
  }
  if (!ok && t == 0) {
    atomicAdd(&g_timeouts, 1ull);
    loss_out[0] = __int_as_float(0x7FC00000);
  }
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    tmem_dealloc(base, T_COLS);
  }
}

// Adam on the mean gradient; c1 = 1 - beta1^step, c2 = 1 - beta2^step
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, float* __restrict__ g,
                       const float* __restrict__ loss, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i] / fmaxf(loss[1], 1.f);
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  g[i] = 0.f;
}

__global__ void k_loss_close(float* loss) {
  loss[2] = loss[0] / fmaxf(loss[1], 1.f);
  loss[0] = 0.f;
  loss[1] = 0.f;
}

// Uniform training pixels: Philox4x32-10, key (seed lo, seed hi), counter (i lo, i hi, 'RCAC', 0)
__global__ void k_random_paths(uint64_t seed, long long n, int W, int H, int base, int32_t* px, int32_t* py,
                               int32_t* ps) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 o = philox10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0x52434143u, 0u), (uint32_t)seed,
                           (uint32_t)(seed >> 32));
  const uint32_t pix = (uint32_t)(((unsigned long long)o.x * (unsigned long long)(W * H)) >> 32);
  px[i] = (int32_t)(pix % (uint32_t)W);
  py[i] = (int32_t)(pix / (uint32_t)W);
  ps[i] = base + (int32_t)i;
}

// Per-pixel sums of the cached frame's path estimates (records' L slots), in sample order
__global__ void k_cache_accum(const float* __restrict__ rec, long long npix, int spp, int W, int H,
                              float* __restrict__ sum, float* __restrict__ sumsq) {
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  float s = 0.f, s2 = 0.f;
  for (int k = 0; k < spp; ++k) {
    const float L = rec[8 * (pix * spp + k) + 7];
    s += L;
    s2 += L * L;
  }
  int px, py;
  render_pixel(pix, W, H, &px, &py);
  const long long p = (long long)py * W + px;
  sum[p] += s;
  if (sumsq) sumsq[p] += s2;
}

int sm_count() {
  int dev = 0, sms = 0;
  TV_CUDA(cudaGetDevice(&dev));
  TV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return sms;
}

template <bool COMPOSE>
void launch_infer(const float* P, float* rec, long long n, float* y, cudaStream_t st) {
  if (n <= 0) return;
  const size_t shm = sizeof(InferSmem);
  // per device and cheap: set on every launch
  TV_CUDA(cudaFuncSetAttribute(k_mlp_infer<COMPOSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  const long long ntiles = (n + MT - 1) / MT;
  long long blocks = sm_count();                 // one block per SM: it holds all 512 TMEM columns
  if (blocks > (ntiles + IG - 1) / IG) blocks = (ntiles + IG - 1) / IG;
  k_mlp_infer<COMPOSE><<<(unsigned)blocks, IG * MT, shm, st>>>(P, rec, n, y);
  TV_LAUNCH();
}

}  // namespace rc
}  // namespace tv

using namespace tv;

extern "C" {

int tg_random_paths(uint64_t seed, int64_t n, int32_t width, int32_t height, int32_t sample_base, int32_t* px,
                    int32_t* py, int32_t* sample, void* cuda_stream) {
  if (n < 0 || width <= 0 || height <= 0 || (long long)width * height > (1ll << 31) || sample_base < 0 ||
      (long long)sample_base + n > (1ll << 31) || (n > 0 && (!px || !py || !sample)))
    return TG_EINVAL;
  if (n == 0) return TG_OK;
  try {
    rc::k_random_paths<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(seed, n, width, height,
                                                                                        sample_base, px, py, sample);
    TV_LAUNCH();
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int tet_cache_samples(const tg_grid* g, const tg_camera* cam, const tg_medium* med, uint64_t seed, int64_t n,
                      const int32_t* px, const int32_t* py, const int32_t* sample, int32_t max_vertices,
                      float* samples, float* L, float survive, int32_t roulette_from, void* cuda_stream) {
  if (!g || !camera_ok(cam) || !medium_ok(med) || n < 0 || max_vertices < 1 || max_vertices > 64 ||
      (n > 0 && (!px || !py || !sample || !samples)) || !(survive >= 0.f && survive <= 1.f) || roulette_from < 0)
    return TG_EINVAL;
  try {
    const GridImpl& G = g->impl;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (n == 0) return TG_OK;
    if (G.n == 0) return TG_EINVAL;
    EstParams ep = est_params(G, *cam, *med, seed);
    ep.spp = 1;
    ep.total = n;
    CallCounter counter(st);
    ep.counter = counter.p;
    ep.px = px; ep.py = py; ep.ps = sample;
    ep.outL = L;
    ep.vtx_cap = max_vertices;
    ep.vtx = samples;
    ep.survive = survive;
    ep.roulette_from = roulette_from;
    run_tet<MODE_TRACE>(G, ep, st);
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int tet_cache_queries(const tg_grid* g, const tg_camera* cam, const tg_medium* med, uint64_t seed, int64_t n,
                      const int32_t* px, const int32_t* py, const int32_t* sample, int32_t cache_depth,
                      float* rec, void* cuda_stream) {
  if (!g || !camera_ok(cam) || !medium_ok(med) || n < 0 || cache_depth < 1 ||
      (n > 0 && (!px || !py || !sample || !rec)))
    return TG_EINVAL;
  try {
    const GridImpl& G = g->impl;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (n == 0) return TG_OK;
    if (G.n == 0) return TG_EINVAL;
    EstParams ep = est_params(G, *cam, *med, seed);
    ep.spp = 1;
    ep.total = n;
    CallCounter counter(st);
    ep.counter = counter.p;
    ep.px = px; ep.py = py; ep.ps = sample;
    ep.cache_depth = cache_depth;
    ep.cache_rec = rec;
    run_tet<MODE_TRACE>(G, ep, st);
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int rc_mlp_infer(const float* params, const float* rec, int64_t n, float* y, void* cuda_stream) {
  if (!params || n < 0 || (n > 0 && (!rec || !y))) return TG_EINVAL;
  try {
    rc::launch_infer<false>(params, const_cast<float*>(rec), n, y, (cudaStream_t)cuda_stream);
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int rc_mlp_grad(const float* params, const float* samples, int64_t n, float* grad, float* loss, void* cuda_stream) {
  if (!params || !grad || !loss || n < 0 || (n > 0 && !samples)) return TG_EINVAL;
  if (reinterpret_cast<uintptr_t>(grad) & 15u) return TG_EINVAL;      // 16-byte atomics into grad
  if (n == 0) return TG_OK;
  try {
    const size_t shm = sizeof(rc::GradSmem);
    TV_CUDA(cudaFuncSetAttribute(rc::k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    const long long ntiles = (n + rc::MT - 1) / rc::MT;
    long long blocks = rc::sm_count();
    if (blocks > ntiles) blocks = ntiles;
    rc::k_mlp_grad<<<(unsigned)blocks, rc::MT, shm, (cudaStream_t)cuda_stream>>>(params, samples, n, grad, loss);
    TV_LAUNCH();
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int rc_adam(float* params, float* m, float* v, float* grad, float* loss, int32_t step, float lr, float beta1,
            float beta2, float eps, void* cuda_stream) {
  if (!params || !m || !v || !grad || !loss || step < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return TG_EINVAL;
  try {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float c1 = (float)(1.0 - std::pow((double)beta1, step));
    const float c2 = (float)(1.0 - std::pow((double)beta2, step));
    rc::k_adam<<<(rc::NPARAM + 255) / 256, 256, 0, st>>>(params, m, v, grad, loss, lr, beta1, beta2, eps, c1, c2);
    TV_LAUNCH();
    rc::k_loss_close<<<1, 1, 0, st>>>(loss);
    TV_LAUNCH();
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int tet_render_cached(const tg_grid* g, const tg_camera* cam, const tg_medium* med, int32_t spp, uint64_t seed,
                      int32_t sample_offset, int32_t cache_depth, const float* params, float* accum_sum,
                      float* accum_sumsq, tg_stats* stats, void* cuda_stream) {
  if (!g || !camera_ok(cam) || !medium_ok(med) || !samples_ok(spp, sample_offset) || cache_depth < 1 || !params ||
      !accum_sum)
    return TG_EINVAL;
  try {
    const GridImpl& G = g->impl;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (spp == 0 || G.n == 0) return TG_OK;
    const long long npix = (long long)cam->width * cam->height;
    const long long total = npix * spp;
    // the frame's path records (32 B each), this call's own
    CallScratch<float> recs((size_t)total * 8, st);
    EstParams ep = est_params(G, *cam, *med, seed);
    ep.spp = spp;
    ep.sample_offset = sample_offset;
    ep.total = total;
    CallCounter counter(st);
    ep.counter = counter.p;
    ep.stats = stats;
    ep.cache_depth = cache_depth;
    ep.cache_rec = recs.p;
    run_tet<MODE_CACHED>(G, ep, st);
    rc::launch_infer<true>(params, recs.p, total, nullptr, st);
    rc::k_cache_accum<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(recs.p, npix, spp, cam->width, cam->height,
                                                                       accum_sum, accum_sumsq);
    TV_LAUNCH();
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int rc_timeouts(int64_t* count) {
  if (!count) return TG_EINVAL;
  unsigned long long c = 0;
  if (cudaMemcpyFromSymbol(&c, rc::g_timeouts, sizeof c) != cudaSuccess) return TG_ECUDA;
  *count = (int64_t)c;
  return TG_OK;
}

}  // extern "C"
