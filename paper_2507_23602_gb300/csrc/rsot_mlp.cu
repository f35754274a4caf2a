// Learned warm start: a small MLP psi_j ~ f(theta, y_j) (density parameters
// theta in R^16, target coordinates y_j in R^2), trained on potentials that
// the solver itself produced.  Layers: in -> W (SiLU) -> W (SiLU) -> W (SiLU)
// -> 1, BF16 weights and activations for the GEMMs, FP32 accumulation, FP32
// master weights and Adam.
//
// GEMM kernel: C[m][n] = sum_k A(m,k) B(n,k) with A(m,k) = A[m*lda+k] or, when
// transposed, A[k*lda+m] (likewise B); CTA tile 128 x 128 x 32, 8 warps of
// 64 x 32, warp-level BF16 tensor-core MMA (m16n8k16, FP32 accumulate),
// operands staged K-contiguous in shared memory (transposed sources are
// transposed on the way in) and read with ldmatrix.  Epilogues: plain FP32,
// bias + SiLU (writes the FP32 pre-activation and the BF16 activation), and
// multiplication by SiLU'(Z) for back-propagation (writes BF16).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rsot_internal.cuh"

namespace rsot {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int GM = 128, GN = 128, GK = 32, GPAD = 8;   // tile, K step, smem row padding
constexpr int G_THREADS = 256;

enum { EPI_F32 = 0, EPI_BIAS_SILU = 1, EPI_DSILU = 2 };

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3,
                                        const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(unsigned &r0, unsigned &r1, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Load a (rows x GK) K-contiguous tile into smem T[rows][GK+GPAD] from either a
// K-contiguous source (src[r*ld + k]) or an r-contiguous one (src[k*ld + r]).
template <bool TRANS, int ROWS>
__device__ __forceinline__ void load_tile(bf16 (*T)[GK + GPAD], const bf16 *__restrict__ src, int ld,
                                          int r0, int rows_total, int k0, int k_total) {
    const bf16 zero = __float2bfloat16(0.0f);
    if (!TRANS) {
        // ROWS * GK / 8 chunks of 8 elements
        for (int c = threadIdx.x; c < ROWS * GK / 8; c += G_THREADS) {
            const int r = c / (GK / 8), kk = (c % (GK / 8)) * 8;
            const int gr = r0 + r, gk = k0 + kk;
            if (gr < rows_total && gk + 8 <= k_total) {
                *reinterpret_cast<uint4 *>(&T[r][kk]) =
                    *reinterpret_cast<const uint4 *>(src + (int64_t)gr * ld + gk);
            } else {
                for (int e = 0; e < 8; ++e)
                    T[r][kk + e] = (gr < rows_total && gk + e < k_total) ? src[(int64_t)gr * ld + gk + e]
                                                                       : zero;
            }
        }
    } else {
        // chunks of 8 consecutive rows at one k
        for (int c = threadIdx.x; c < ROWS * GK / 8; c += G_THREADS) {
            const int kk = c / (ROWS / 8), r = (c % (ROWS / 8)) * 8;
            const int gr = r0 + r, gk = k0 + kk;
            bf16 v[8];
            if (gk < k_total && gr + 8 <= rows_total) {
                *reinterpret_cast<uint4 *>(v) =
                    *reinterpret_cast<const uint4 *>(src + (int64_t)gk * ld + gr);
            } else {
                for (int e = 0; e < 8; ++e)
                    v[e] = (gk < k_total && gr + e < rows_total) ? src[(int64_t)gk * ld + gr + e] : zero;
            }
            for (int e = 0; e < 8; ++e) T[r + e][kk] = v[e];
        }
    }
}

template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(G_THREADS)
    k_gemm_bf16(int M, int N, int K, int kslice, const bf16 *__restrict__ A, int lda,
                const bf16 *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                const float *__restrict__ bias, bf16 *__restrict__ H, int ldh, bf16 *__restrict__ Z,
                int ldz) {
    __shared__ __align__(16) bf16 As[GM][GK + GPAD];
    __shared__ __align__(16) bf16 Bs[GN][GK + GPAD];
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 2) * 64, wn = (warp & 3) * 32;   // 2 x 4 warps of 64 x 32
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    // split K: slice z covers [z kslice, (z + 1) kslice) and writes its own partial C
    const int kb = blockIdx.z * kslice, ke = min(K, kb + kslice);
    if (EPI == EPI_F32) C += (int64_t)blockIdx.z * M * ldc;
    for (int k0 = kb; k0 < ke; k0 += GK) {
        load_tile<AT, GM>(As, A, lda, m0, M, k0, ke);
        load_tile<BT, GN>(Bs, B, ldb, n0, N, k0, ke);
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GK; ks += 16) {
            unsigned a[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = wm + i * 16 + (lane & 15);
                const int c = ks + (lane >> 4) * 8;
                ldsm_x4(a[i][0], a[i][1], a[i][2], a[i][3], &As[r][c]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                unsigned b0, b1;
                const int r = wn + j * 8 + (lane & 7);
                const int c = ks + ((lane >> 3) & 1) * 8;
                ldsm_x2(b0, b1, &Bs[r][c]);
#pragma unroll
                for (int i = 0; i < 4; ++i) mma_bf16(acc[i][j], a[i], b0, b1);
            }
        }
        __syncthreads();
    }
    // epilogue
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm + i * 16 + g + h * 8;
                const int col = n0 + wn + j * 8 + t4 * 2;
                if (row >= M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int cc = col + e;
                    if (cc >= N) continue;
                    float v = acc[i][j][h * 2 + e];
                    if (EPI == EPI_F32) {
                        C[(int64_t)row * ldc + cc] = v;
                    } else if (EPI == EPI_BIAS_SILU) {
                        v += bias[cc];
                        Z[(int64_t)row * ldz + cc] = __float2bfloat16(v);       // pre-activation
                        H[(int64_t)row * ldh + cc] = __float2bfloat16(silu(v));  // activation
                    } else {
                        H[(int64_t)row * ldh + cc] =
                            __float2bfloat16(v * dsilu(__bfloat162float(Z[(int64_t)row * ldz + cc])));
                    }
                }
            }
}

// ---------------------------------------------------------------------------
// The same GEMM on the fifth-generation tensor cores.  One thread issues
// tcgen05.mma (kind::f16: BF16 operands, FP32 accumulator in tensor memory),
// CTA tile 128 x 128 (256 threads), K in stages of 64 (four MMAs of K = 16),
// two stages in shared memory: the MMAs of a stage are issued as soon as its
// operands have landed, and the next stage is copied while they run (into the
// other buffer, once the commit of the MMAs that last read it has arrived).
// Operands sit in the canonical K-major layout without swizzle: 8 x 8 core
// matrices (8 rows of 16 bytes, 128 contiguous bytes), consecutive along K
// (LBO = 128 B), 8-row groups 1,040 B apart (SBO), so a stage tile of 128 rows
// x 64 K takes 16,640 B and no descriptor offset can leave it.  K-contiguous sources
// arrive by 16-byte cp.async (zero-filled outside the matrix); a transposed
// source is transposed on the way in by the threads.  A K-contiguous operand
// whose rows start on 16-byte boundaries comes instead by one TMA tile copy
// per stage (tensor map box of 64 K x 128 rows, zero-filled outside the
// matrix, 128-byte swizzle): rows of 128 B in 8-row atoms of 1,024 B (SBO),
// the 16-byte chunks of row r permuted by r % 8, which the MMA's descriptor
// (swizzle mode 128 B) undoes; the K = 16 steps advance its start address by
// 32 B inside the atom.  A transposed operand (MN contiguous) comes by two TMA
// copies of 64 MN x 64 K (8 KB apart) and is read MN-major (transpose bit of
// the instruction descriptor): 128-byte rows along MN, one per k, 8-row atoms
// 1,024 B apart along K (SBO), the two 64-wide MN halves 8,192 B apart (LBO),
// 2,048 B per K = 16 step.  The accumulator (128
// lanes x 128 FP32 columns) is read back by tcgen05.ld: warp w takes lanes
// 32 (w % 4) .. + 31 and columns 64 (w / 4) .. + 63, transposes each 32 x 32
// block through shared memory and stores whole rows (coalesced), for the
// epilogues of the warp-level kernel above.  Every wait is bounded (flag
// kErrTimeout).
constexpr int T5_M = 128, T5_N = 128, T5_K = 64, T5_THREADS = 256;
// 8-row groups 1,040 B apart (1,024 + 16: successive groups start in other
// shared-memory banks, for the transposing loads)
constexpr uint32_t T5_LBO = 128, T5_SBO = 1040;
constexpr int T5_TILE = 16 * T5_SBO;       // bytes of one cp.async operand tile (16 row groups)
constexpr int T5_TILE_TMA = 128 * 128;     // bytes of one TMA operand tile (128 rows of 128 B)
constexpr int T5_TS = 17 * 1024;           // operand slot: holds either tile, 1,024-aligned
constexpr int T5_SMEM = 2 * 2 * T5_TS + 1024;   // two stages of A and B, alignment slack: 69 KB
static_assert(T5_TILE <= T5_TS && T5_TILE_TMA <= T5_TS, "operand tiles fit their slots");
static_assert(T5_THREADS / 32 * 32 * 33 * 4 <= 4 * T5_TS, "epilogue transpose fits in the stage buffers");
// instruction descriptor of kind::f16: F32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t T5_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(T5_N >> 3) << 17) |
                              ((uint32_t)(T5_M >> 4) << 24);

// shared-memory matrix descriptor: start address >> 4 (bits 0-13), LBO >> 4
// (bits 16-29), SBO >> 4 (bits 32-45), the fixed value 1 at bits 46-48, base
// offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(T5_LBO >> 4) << 16) |
           ((uint64_t)(T5_SBO >> 4) << 32) | (1ull << 46);
}
// the same for a TMA tile: SBO 1,024 B (8-row atoms), LBO unused within one
// 128-byte row (encoded 1), swizzle mode 2 (128 B) at bits 61-63
__device__ __forceinline__ uint64_t t5_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}
// an MN-major TMA tile: LBO 8,192 B (the two 64-wide MN halves), SBO 1,024 B
// (8 k-rows of 128 B), swizzle mode 2
__device__ __forceinline__ uint64_t t5_desc_mn_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(8192 >> 4) << 16) |
           ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// one 2-D TMA tile copy global -> shared (x = K element, y = row), completion
// counted in bytes on bar
__device__ __forceinline__ void tma_load_2d(void *smem, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(smem)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// one 2-D TMA tile copy shared -> global (x = column, y = row) in the thread's
// bulk group; the part of the box beyond the tensor's extent is not written
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *smem, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(smem)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the bulk group's reads of shared memory are done (its global writes complete
// on their own; the kernel's end orders them before later work on the stream)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, unsigned bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// element (r, k) of a 128 x 64 stage tile at byte (r / 8) SBO + (k / 8) LBO +
// (r % 8) 16 + (k % 8) 2; rows r0 + r >= rows_total and k0 + k >= k_total are zero
template <bool TRANS>
__device__ __forceinline__ void t5_load(unsigned char *T, const bf16 *__restrict__ src, int ld, int r0,
                                        int rows_total, int k0, int k_total) {
    const bf16 zero = __float2bfloat16(0.0f);
    if (!TRANS) {
        // src[r * ld + k]: 16-byte chunks of 8 consecutive k, asynchronous (zero-filled
        // when the chunk lies outside; a chunk cut by k_total is assembled here)
        for (int c = threadIdx.x; c < 128 * (T5_K / 8); c += T5_THREADS) {
            const int r = c / (T5_K / 8), kc = c % (T5_K / 8);
            const int gr = r0 + r, gk = k0 + kc * 8;
            unsigned char *dst = T + (r >> 3) * T5_SBO + kc * T5_LBO + (r & 7) * 16;
            if (gr < rows_total && gk < k_total && gk + 8 > k_total) {
                bf16 e[8];
                for (int i = 0; i < 8; ++i) e[i] = gk + i < k_total ? src[(int64_t)gr * ld + gk + i] : zero;
                *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(e);
            } else {
                const bool in = gr < rows_total && gk + 8 <= k_total;
                cp_async16(dst, in ? (const void *)(src + (int64_t)gr * ld + gk) : (const void *)src,
                           in ? 16u : 0u);
            }
        }
    } else {
        // src[k * ld + r]: 8 consecutive rows at one k per load, spread over one 8-row group
        for (int c = threadIdx.x; c < 128 * T5_K / 8; c += T5_THREADS) {
            const int k = c / 16, rg = c % 16;
            const int gk = k0 + k, gr = r0 + rg * 8;
            bf16 v[8];
            if (gk < k_total && gr + 8 <= rows_total) {
                *reinterpret_cast<uint4 *>(v) = *reinterpret_cast<const uint4 *>(src + (int64_t)gk * ld + gr);
            } else {
                for (int i = 0; i < 8; ++i)
                    v[i] = (gk < k_total && gr + i < rows_total) ? src[(int64_t)gk * ld + gr + i] : zero;
            }
            unsigned char *base = T + rg * T5_SBO + (k >> 3) * T5_LBO + (k & 7) * 2;
            for (int i = 0; i < 8; ++i) *reinterpret_cast<bf16 *>(base + i * 16) = v[i];
        }
    }
}

// 32 consecutive FP32 columns of the thread's tensor-memory lane
__device__ __forceinline__ void t5_ld32(uint32_t (&v)[32], uint32_t taddr) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(T5_THREADS)
    k_gemm_t5(int M, int N, int K, int kslice, const bf16 *__restrict__ A, int lda,
              const bf16 *__restrict__ B, int ldb, float *__restrict__ C, int ldc, const float *__restrict__ bias,
              bf16 *__restrict__ H, int ldh, bf16 *__restrict__ Z, int ldz,
              int *__restrict__ flags, const __grid_constant__ CUtensorMap tmA,
              const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmH,
              const __grid_constant__ CUtensorMap tmZ, int tma) {
    extern __shared__ __align__(1024) unsigned char t5_dyn[];
    __shared__ __align__(8) uint64_t done[2];   // commit of the MMAs that read stage buffer s
    __shared__ __align__(8) uint64_t full[2];   // TMA bytes of stage buffer s have landed
    __shared__ uint32_t s_tmem;
    __shared__ float s_bias[T5_N];
    // operand slots on 1,024-byte boundaries (the 128-byte swizzle atoms)
    unsigned char *const t5_smem = t5_dyn + ((1024u - (smem_u32(t5_dyn) & 1023u)) & 1023u);
    // tma bit 0: A by TMA, bit 1: B by TMA; a transposed operand copied by TMA
    // is read MN-major (transpose bits 15 / 16 of the instruction descriptor);
    // bit 2: H stored by TMA, bit 3: Z stored by TMA (BF16 epilogues)
    const bool tA = (tma & 1) != 0, tB = (tma & 2) != 0;
    const unsigned tx = (tA ? T5_TILE_TMA : 0) + (tB ? T5_TILE_TMA : 0);
    const uint32_t idesc = T5_IDESC | ((tA && AT) ? 1u << 15 : 0u) | ((tB && BT) ? 1u << 16 : 0u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * T5_M, n0 = blockIdx.x * T5_N;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(T5_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (EPI == EPI_BIAS_SILU)
        for (int i = tid; i < T5_N; i += T5_THREADS) s_bias[i] = n0 + i < N ? bias[n0 + i] : 0.f;
    if (tid == 32) {
        mbar_init(&done[0], 1);
        mbar_init(&done[1], 1);
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_barrier_init();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    if (EPI == EPI_DSILU && warp == 7 && (N - n0) % 8 == 0 && ldz % 8 == 0) {
        // the epilogue's Z rows go to L2 while the MMAs run: one bulk prefetch per
        // row of the tile (min(T5_N, N - n0) BF16 = a multiple of 16 bytes, and
        // row starts on 16-byte boundaries since ldz and n0 are multiples of 8)
        const unsigned bytes = (unsigned)min(T5_N, N - n0) * 2u;
        for (int i = lane; i < T5_M && m0 + i < M; i += 32)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Z + (int64_t)(m0 + i) * ldz + n0),
                         "r"(bytes)
                         : "memory");
    }
    // split K: slice z covers [z kslice, (z + 1) kslice) and writes its own partial C
    const int kb = blockIdx.z * kslice, ke = min(K, kb + kslice);
    if (EPI == EPI_F32) C += (int64_t)blockIdx.z * M * ldc;
    const int nk = ke > kb ? (ke - kb + T5_K - 1) / T5_K : 0;
    bool ok = true;
    // stage loader: TMA operands by thread 0 (the tensor map zero-fills rows and
    // K beyond the matrix; the host takes TMA only when the K slice is all of K),
    // the others by every thread's cp.async
    auto load_stage = [&](int buf, int k0) {
        unsigned char *As = t5_smem + buf * 2 * T5_TS, *Bs = As + T5_TS;
        if (tx && tid == 0) {
            mbar_expect_tx(&full[buf], tx);
            if (tA) {
                if (AT) {
                    tma_load_2d(As, &tmA, m0, k0, &full[buf]);
                    tma_load_2d(As + T5_TILE_TMA / 2, &tmA, m0 + 64, k0, &full[buf]);
                } else {
                    tma_load_2d(As, &tmA, k0, m0, &full[buf]);
                }
            }
            if (tB) {
                if (BT) {
                    tma_load_2d(Bs, &tmB, n0, k0, &full[buf]);
                    tma_load_2d(Bs + T5_TILE_TMA / 2, &tmB, n0 + 64, k0, &full[buf]);
                } else {
                    tma_load_2d(Bs, &tmB, k0, n0, &full[buf]);
                }
            }
        }
        if (!tA) t5_load<AT>(As, A, lda, m0, M, k0, ke);
        if (!tB) t5_load<BT>(Bs, B, ldb, n0, N, k0, ke);
        cp_async_commit();
    };
    // thread 0: bit s of fbad = a TMA wait of buffer s gave up, bit s of fpar =
    // parity of buffer s's next completion
    unsigned fbad = 0u, fpar = 0u;
    if (nk > 0) load_stage(0, kb);
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt & 1;
        unsigned char *As = t5_smem + s * 2 * T5_TS, *Bs = As + T5_TS;
        // stage kt has landed (the thread's copies, then every thread's); its
        // stores become visible to the tensor core (async proxy)
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            if (tx) {
                const bool got = mbar_wait(&full[s], (fpar >> s) & 1u);
                fbad = got ? fbad & ~(1u << s) : fbad | (1u << s);
                ok = got && ok;
                fpar ^= 1u << s;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
            for (int kk = 0; kk < T5_K / 16; ++kk) {
                const uint64_t ad = !tA ? t5_desc(a0 + kk * 2 * T5_LBO)
                                    : AT ? t5_desc_mn_sw128(a0 + kk * 2048) : t5_desc_sw128(a0 + kk * 32);
                const uint64_t bd = !tB ? t5_desc(b0 + kk * 2 * T5_LBO)
                                    : BT ? t5_desc_mn_sw128(b0 + kk * 2048) : t5_desc_sw128(b0 + kk * 32);
                const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&done[s]))
                         : "memory");
        }
        if (kt + 1 < nk) {
            // the other buffer was last read by the MMAs of stage kt - 1
            if (kt >= 1) ok = mbar_wait(&done[s ^ 1], (unsigned)((kt - 1) >> 1) & 1u) && ok;
            load_stage(s ^ 1, kb + (kt + 1) * T5_K);
        }
    }
    if (nk > 0) ok = mbar_wait(&done[(nk - 1) & 1], (unsigned)((nk - 1) >> 1) & 1u) && ok;
    // a TMA wait that gave up may leave its copy in flight: wait for it once
    // more (bounded) before the buffers are reused or the CTA exits
    if (tid == 0 && tx)
        for (int b = 0; b < 2; ++b)
            if ((fbad >> b) & 1u) mbar_wait(&full[b], ((fpar >> b) & 1u) ^ 1u);
    // one verdict for the CTA: a wait that gave up in any thread voids the tile
    // (and raises the flag below); the shared-memory epilogue starts after
    // thread 0's last wait for its copies
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int q = warp & 3, cb = (warp >> 2) * 64;   // lanes 32 q .. + 31, columns cb .. + 63
    const bool tstore = EPI != EPI_F32 && (tma & 4) && (EPI != EPI_BIAS_SILU || (tma & 8));
    if (tstore) {
        // BF16 epilogue through TMA stores: every MMA is done, so the stage buffers
        // hold the output tiles, per 64 columns a box of 128 rows x 128 B in the
        // 128-byte swizzle (16-byte chunk j of row r at chunk j ^ (r % 8)): H at 0
        // and 16 KB, Z at 32 and 48 KB.  The thread owns TMEM lane (row) r and
        // writes whole 16-byte chunks (eight lanes of a quarter-warp: eight
        // different chunk positions, no bank conflict)
        unsigned char *const sH = t5_smem, *const sZ = t5_smem + 32768;
        const int r = 32 * q + lane;
        const bool live = ok && nk > 0;
#pragma unroll 1
        for (int c0 = cb; c0 < cb + 64; c0 += 32) {
            uint32_t v[32];
            t5_ld32(v, tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0);
            const int hb = (c0 >> 6) * 16384, ch0 = (c0 & 63) >> 3;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int cc = c0 + 8 * k;   // first column of the chunk within the tile
                const unsigned off = (unsigned)(hb + r * 128 + (((ch0 + k) ^ (r & 7)) << 4));
                uint4 hv;
                if (EPI == EPI_BIAS_SILU) {
                    uint4 zv;
                    float x[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = __uint_as_float(v[8 * k + i]) + s_bias[cc + i];
                    zv.x = pack_bf16(x[0], x[1]);    // pre-activation
                    zv.y = pack_bf16(x[2], x[3]);
                    zv.z = pack_bf16(x[4], x[5]);
                    zv.w = pack_bf16(x[6], x[7]);
                    hv.x = pack_bf16(silu(x[0]), silu(x[1]));   // activation
                    hv.y = pack_bf16(silu(x[2]), silu(x[3]));
                    hv.z = pack_bf16(silu(x[4]), silu(x[5]));
                    hv.w = pack_bf16(silu(x[6]), silu(x[7]));
                    *reinterpret_cast<uint4 *>(sZ + off) = zv;
                } else {
                    // x SiLU'(Z) with the stored BF16 pre-activation of the row
                    uint4 zin = make_uint4(0u, 0u, 0u, 0u);
                    if (live && m0 + r < M && n0 + cc < N)
                        zin = *reinterpret_cast<const uint4 *>(Z + (int64_t)(m0 + r) * ldz + n0 + cc);
                    const __nv_bfloat162 *z2 = reinterpret_cast<const __nv_bfloat162 *>(&zin);
                    uint32_t *hp = &hv.x;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 z = __bfloat1622float2(z2[i]);
                        hp[i] = pack_bf16(__uint_as_float(v[8 * k + 2 * i]) * dsilu(z.x),
                                          __uint_as_float(v[8 * k + 2 * i + 1]) * dsilu(z.y));
                    }
                }
                *reinterpret_cast<uint4 *>(sH + off) = hv;
            }
        }
        // the tiles' generic-proxy writes become visible to the TMA (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && live) {
            for (int h = 0; h < 2; ++h)
                if (n0 + 64 * h < N) {
                    tma_store_2d(&tmH, sH + h * 16384, n0 + 64 * h, m0);
                    if (EPI == EPI_BIAS_SILU) tma_store_2d(&tmZ, sZ + h * 16384, n0 + 64 * h, m0);
                }
            bulk_commit();
            bulk_wait_read();   // the tiles have left shared memory before the CTA exits
        }
    }
    // every MMA is done: the stage buffers hold the epilogue's transposes
    float *T = reinterpret_cast<float *>(t5_smem) + warp * 32 * 33;
#pragma unroll 1
    for (int c0 = cb; c0 < (tstore ? cb : cb + 64); c0 += 32) {
        uint32_t v[32];
        t5_ld32(v, tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0);
#pragma unroll
        for (int j = 0; j < 32; ++j) T[lane * 33 + j] = __uint_as_float(v[j]);
        __syncwarp();
        const int col = n0 + c0 + lane;
        if (ok && nk > 0 && col < N) {
            const float bc = EPI == EPI_BIAS_SILU ? bias[col] : 0.f;
            // eight rows at a time: their SiLU'(Z) operands are loaded before the stores
#pragma unroll 1
            for (int r8 = 0; r8 < 32; r8 += 8) {
                float zr[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int row = m0 + 32 * q + r8 + i;
                    zr[i] = (EPI == EPI_DSILU && row < M) ? __bfloat162float(Z[(int64_t)row * ldz + col]) : 0.f;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int row = m0 + 32 * q + r8 + i;
                    if (row >= M) break;
                    float x = T[(r8 + i) * 33 + lane];
                    if (EPI == EPI_F32) {
                        C[(int64_t)row * ldc + col] = x;
                    } else if (EPI == EPI_BIAS_SILU) {
                        x += bc;
                        Z[(int64_t)row * ldz + col] = __float2bfloat16(x);      // pre-activation
                        H[(int64_t)row * ldh + col] = __float2bfloat16(silu(x));  // activation
                    } else {
                        H[(int64_t)row * ldh + col] = __float2bfloat16(x * dsilu(zr[i]));
                    }
                }
            }
        }
        __syncwarp();
    }
    if (!ok && tid == 0) atomicOr(flags, kErrTimeout);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T5_N) : "memory");
}

// ------------------------------------------------ persistent tcgen05 GEMM (t6)
// The BF16-epilogue GEMMs of the network (forward: bias + SiLU; back-
// propagation: x SiLU'(Z)) with K-contiguous A [M][K] and B [N][K], N <= 256
// a multiple of 32: one CTA per SM loops over 128-row tiles, each covering all
// N columns, with warp-specialised roles so that a tile's epilogue overlaps the
// next tile's MMAs:
//   warp 0 (one lane): TMA copies of A (64 K x 128 rows) and B (64 K x N rows),
//     128-byte swizzle, into T6_STAGES stages (full / empty mbarriers);
//   warp 1: allocates 2 N TMEM columns (two accumulators); one lane issues
//     tcgen05.mma (M 128, N, K 16) and commits each stage back to its empty
//     barrier and each finished tile to its accumulator's full barrier;
//   warps 2-17: the epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31 (its
//     rows) and the box of 64 columns 64 (w - 2) / 4;
//     it releases the accumulator after its last tcgen05.ld and stores each
//     box (32 rows x 64 columns) through its staging tile in the 128-byte
//     swizzle (TMA stores by the warp's lane 0); for x SiLU'(Z) the warp's Z
//     box comes by TMA into the same layout while the tile's MMAs run.  Four
//     warps per lane quarter keep the conversions and SiLU evaluations up with
//     the MMAs (with one or two per quarter the epilogue was the bottleneck).
// Every mbarrier wait is bounded; a wait that gives up raises kErrTimeout and
// its role stops (the others then give up on their own waits).
constexpr int T6_STAGES = 2, T6_EPI = 16, T6_THREADS = 32 * (2 + T6_EPI);
constexpr int T6_A = 128 * 128;                     // A stage: 128 rows x 128 B
constexpr int T6_B = 256 * 128;                     // B stage: up to 256 rows x 128 B
constexpr int T6_STAGE = T6_A + T6_B;
constexpr int T6_BOX = 32 * 128;                    // staging box: 32 rows x 64 BF16 columns
constexpr int T6_STG = T6_EPI * 2 * T6_BOX;         // per epilogue warp: H and Z boxes
constexpr int T6_SMEM = T6_STAGES * T6_STAGE + T6_STG + 1024;   // + alignment slack: 225 KB
static_assert(T6_SMEM + 2048 <= 232448, "the persistent GEMM's shared memory fits one CTA per SM");

__device__ __forceinline__ void tcgen05_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(T6_THREADS, 1)
    k_gemm_t6(int M, int N, int K, int kslice, int mblocks, float *__restrict__ C, int ldc,
              const float *__restrict__ bias, int *__restrict__ flags, const __grid_constant__ CUtensorMap tmA,
              const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmH,
              const __grid_constant__ CUtensorMap tmZ) {
    extern __shared__ __align__(1024) unsigned char t6_dyn[];
    __shared__ __align__(8) uint64_t full[T6_STAGES], empty[T6_STAGES], accf[2], acce[2], mdone, zbar[T6_EPI];
    __shared__ uint32_t s_tmem;
    __shared__ float s_bias[256];
    unsigned char *const sm = t6_dyn + ((1024u - (smem_u32(t6_dyn) & 1023u)) & 1023u);
    unsigned char *const stg = sm + T6_STAGES * T6_STAGE;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tile t: rows 128 (t % mblocks) .., K slice t / mblocks (partials at C + slice M ldc)
    const int tiles = mblocks * ((K + kslice - 1) / kslice);
    auto tile_rows = [&](int t) { return (t % mblocks) * 128; };
    auto tile_k0 = [&](int t) { return (t / mblocks) * kslice; };
    auto tile_nkb = [&](int t) { return (min(K, tile_k0(t) + kslice) - tile_k0(t) + 63) / 64; };
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (AT ? 1u << 15 : 0u) | (BT ? 1u << 16 : 0u) |
                           ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t tcols = N <= 16 ? 32u : N <= 32 ? 64u : N <= 64 ? 128u : N <= 128 ? 256u : 512u;
    if (EPI == EPI_BIAS_SILU)
        for (int i = tid; i < 256; i += T6_THREADS) s_bias[i] = i < N ? bias[i] : 0.f;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < T6_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], T6_EPI);
        }
        mbar_init(&mdone, 1);
        for (int e = 0; e < T6_EPI; ++e) mbar_init(&zbar[e], 1);
        fence_barrier_init();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    bool ok = true;
    if (warp == 0) {
        // producer: stage it % T6_STAGES, its n-th use waits for the (n - 1)-th release
        if (lane == 0) {
            // A: one box of 64 K x 128 rows, or transposed two of 64 rows x 64 K
            // (8 KB apart, read MN-major); B: one box of 64 K x N rows, or
            // transposed N / 64 boxes of 64 columns x 64 K
            const unsigned bytes = (unsigned)(T6_A + (BT ? (N + 63) / 64 * 8192 : N * 128));
            int it = 0;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const int m0 = tile_rows(t), kb0 = tile_k0(t), nkb = tile_nkb(t);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % T6_STAGES, n = it / T6_STAGES;
                    if (n > 0 && !mbar_wait(&empty[s], (unsigned)(n - 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    unsigned char *As = sm + s * T6_STAGE, *Bs = As + T6_A;
                    const int k0 = kb0 + 64 * kb;
                    mbar_expect_tx(&full[s], bytes);
                    if (AT) {
                        tma_load_2d(As, &tmA, m0, k0, &full[s]);
                        tma_load_2d(As + 8192, &tmA, m0 + 64, k0, &full[s]);
                    } else {
                        tma_load_2d(As, &tmA, k0, m0, &full[s]);
                    }
                    if (BT)
                        for (int i = 0; 64 * i < N; ++i) tma_load_2d(Bs + 8192 * i, &tmB, 64 * i, k0, &full[s]);
                    else
                        tma_load_2d(Bs, &tmB, k0, 0, &full[s]);
                }
            }
            // copies still in flight land before the CTA exits: the last copy into
            // every stage is awaited (bounded)
            for (int s = 0; s < T6_STAGES; ++s) {
                const int uses = it / T6_STAGES + (s < it % T6_STAGES ? 1 : 0);
                if (uses > 0) (void)mbar_wait(&full[s], (unsigned)(uses - 1) & 1u);
            }
            if (!ok) atomicOr(flags, kErrTimeout);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, tc = 0;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++tc) {
                const int a = tc & 1, na = tc >> 1;
                if (na > 0 && !mbar_wait(&acce[a], (unsigned)(na - 1) & 1u)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int nkb = tile_nkb(t);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % T6_STAGES, n = it / T6_STAGES;
                    if (!mbar_wait(&full[s], (unsigned)n & 1u)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(sm + s * T6_STAGE), b0 = a0 + T6_A;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = AT ? t5_desc_mn_sw128(a0 + kk * 2048) : t5_desc_sw128(a0 + kk * 32);
                        const uint64_t bd = BT ? t5_desc_mn_sw128(b0 + kk * 2048) : t5_desc_sw128(b0 + kk * 32);
                        const uint32_t accum = (kb > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                tmem + (uint32_t)(a * N)),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                            : "memory");
                    }
                    tcgen05_commit(&empty[s]);   // the stage is free once these MMAs are done
                }
                if (!ok) break;
                tcgen05_commit(&accf[a]);        // the tile's accumulator is complete
            }
            // every MMA issued is complete before the tensor memory is freed
            tcgen05_commit(&mdone);
            (void)mbar_wait(&mdone, 0u);
            if (!ok) atomicOr(flags, kErrTimeout);
        }
    } else {
        // epilogue warps: rows 32 q .. + 31 of each tile, boxes 64 (jb + T6_EPI / 4 i)
        const int q = warp & 3, jb = (warp - 2) >> 2;
        unsigned char *const bH = stg + (warp - 2) * (2 * T6_BOX), *const bZ = bH + T6_BOX;
        // x SiLU'(Z): the warp's Z box (32 rows x 64 columns, at most one per tile
        // since N <= 256) comes by TMA into its Z staging tile while the MMAs run
        const int cz = 64 * jb, e = warp - 2;
        int tc = 0, nz = 0;
        bool zpend = false;
        for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++tc) {
            const int a = tc & 1, na = tc >> 1, m0 = tile_rows(t);
            if (EPI == EPI_DSILU && cz < N && lane == 0) {
                mbar_expect_tx(&zbar[e], (unsigned)T6_BOX);
                tma_load_2d(bZ, &tmZ, cz, m0 + 32 * q, &zbar[e]);
                zpend = true;
            }
            if (!__all_sync(0xffffffffu, mbar_wait(&accf[a], (unsigned)na & 1u))) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (EPI == EPI_DSILU && cz < N) {
                if (!__all_sync(0xffffffffu, mbar_wait(&zbar[e], (unsigned)nz & 1u))) {
                    ok = false;
                    break;
                }
                ++nz;
                zpend = false;
            }
            for (int cb = 64 * jb; cb < N; cb += 64 * (T6_EPI / 4)) {
                if constexpr (EPI == EPI_F32) {
                    // FP32 (split-K partials of the slice, rows slice M + row of the
                    // partials' map): two boxes of 32 columns x the warp's 32 rows in
                    // the staging tiles (16-byte chunk j of row r at j ^ (r % 8)),
                    // stored by TMA; M is a multiple of 32, so a box never reaches
                    // into the next slice's rows
                    const int prow = (t / mblocks) * M + m0 + 32 * q;
                    const bool rows_in = m0 + 32 * q < M;
#pragma unroll 1
                    for (int hf = 0; hf < 2 && cb + 32 * hf < N; ++hf) {
                        const int c0 = cb + 32 * hf;
                        uint32_t v[32];
                        t5_ld32(v, tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * N + c0));
                        if (hf == 0) {
                            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                            __syncwarp();
                        }
                        unsigned char *const bx = hf ? bZ : bH;
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            *reinterpret_cast<uint4 *>(bx + lane * 128 + ((i ^ (lane & 7)) << 4)) =
                                make_uint4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0 && rows_in) {
                        tma_store_2d(&tmH, bH, cb, prow);
                        if (cb + 32 < N) tma_store_2d(&tmH, bZ, cb + 32, prow);
                        bulk_commit();
                    }
                } else {
#pragma unroll 1
                for (int hf = 0; hf < 2 && cb + 32 * hf < N; ++hf) {
                    const int c0 = cb + 32 * hf;
                    uint32_t v[32];
                    t5_ld32(v, tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * N + c0));
                    uint4 hv[4], zv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int cc = c0 + 8 * k;
                        if (EPI == EPI_BIAS_SILU) {
                            float x[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) x[i] = __uint_as_float(v[8 * k + i]) + s_bias[cc + i];
                            zv[k].x = pack_bf16(x[0], x[1]);
                            zv[k].y = pack_bf16(x[2], x[3]);
                            zv[k].z = pack_bf16(x[4], x[5]);
                            zv[k].w = pack_bf16(x[6], x[7]);
                            hv[k].x = pack_bf16(silu(x[0]), silu(x[1]));
                            hv[k].y = pack_bf16(silu(x[2]), silu(x[3]));
                            hv[k].z = pack_bf16(silu(x[4]), silu(x[5]));
                            hv[k].w = pack_bf16(silu(x[6]), silu(x[7]));
                        } else {
                            // Z of the row from the swizzled staging tile (zero beyond M)
                            const uint4 zin = *reinterpret_cast<const uint4 *>(
                                bZ + lane * 128 + (((4 * hf + k) ^ (lane & 7)) << 4));
                            const __nv_bfloat162 *z2 = reinterpret_cast<const __nv_bfloat162 *>(&zin);
                            uint32_t *hp = &hv[k].x;
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const float2 z = __bfloat1622float2(z2[i]);
                                hp[i] = pack_bf16(__uint_as_float(v[8 * k + 2 * i]) * dsilu(z.x),
                                                  __uint_as_float(v[8 * k + 2 * i + 1]) * dsilu(z.y));
                            }
                        }
                    }
                    if (hf == 0) {
                        // the previous box's store has read the staging tile
                        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                        __syncwarp();
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const unsigned off = (unsigned)(lane * 128 + (((4 * hf + k) ^ (lane & 7)) << 4));
                        *reinterpret_cast<uint4 *>(bH + off) = hv[k];
                        if (EPI == EPI_BIAS_SILU) *reinterpret_cast<uint4 *>(bZ + off) = zv[k];
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    tma_store_2d(&tmH, bH, cb, m0 + 32 * q);
                    if (EPI == EPI_BIAS_SILU) tma_store_2d(&tmZ, bZ, cb, m0 + 32 * q);
                    bulk_commit();
                }
                }
            }
            // every TMEM read of this accumulator by the warp is done: release it
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[a]);
        }
        if (lane == 0) bulk_wait_read();
        // a Z copy issued before a wait that gave up lands before the CTA exits
        if (zpend && lane == 0) (void)mbar_wait(&zbar[e], (unsigned)nz & 1u);
        if (!ok && lane == 0) atomicOr(flags, kErrTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// out[b] = sum_i H3[b][i] w4[i] + b4 (FP32), one warp per row; for widths of
// at most 256 (a multiple of 8) lane l takes columns 8l .. 8l + 7 in one
// 16-byte load
__global__ void k_head_v8(const bf16 *__restrict__ H, int width, int64_t rows, const float *__restrict__ w,
                          const float *__restrict__ b, float *__restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float s = 0.f;
    if (8 * lane < width) {
        const uint4 hv = *reinterpret_cast<const uint4 *>(H + r * width + 8 * lane);
        const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&hv);
        const float4 wa = *reinterpret_cast<const float4 *>(w + 8 * lane);
        const float4 wb = *reinterpret_cast<const float4 *>(w + 8 * lane + 4);
        const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 hf = __bfloat1622float2(h2[k]);
            s = fmaf(hf.x, wv[2 * k], s);
            s = fmaf(hf.y, wv[2 * k + 1], s);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s + b[0];
}
// out[b] = sum_i H3[b][i] w4[i] + b4 (FP32), one warp per row
__global__ void k_head(const bf16 *__restrict__ H, int width, int64_t rows, const float *__restrict__ w,
                       const float *__restrict__ b, float *__restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float s = 0.f;
    for (int i = lane; i < width; i += 32) s += __bfloat162float(H[r * width + i]) * w[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s + b[0];
}

// d_out = (out - y) / B (loss = mean (out - y)^2 / 2), per-row loss terms;
// dZ3 = d_out w4 * SiLU'(Z3) (BF16)
__global__ void k_head_back(const float *__restrict__ out, const float *__restrict__ y, int64_t rows,
                            int64_t valid, float inv_b, const float *__restrict__ w4,
                            const bf16 *__restrict__ Z3, int width, float *__restrict__ dout,
                            bf16 *__restrict__ dZ3, float *__restrict__ loss_terms) {
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const float e = r < valid ? out[r] - y[r] : 0.f;
    const float d = e * inv_b;
    if (lane == 0) {
        dout[r] = d;
        loss_terms[r] = 0.5f * e * e;
    }
    for (int i = lane; i < width; i += 32)
        dZ3[r * width + i] = __float2bfloat16(d * w4[i] * dsilu(__bfloat162float(Z3[r * width + i])));
}

// The head's back-propagation with its column sums, for widths of at most 256
// (a multiple of 8): per row d_out = (out - y) / B and its loss term, dZ3 =
// BF16(d_out w4 SiLU'(Z3)), and per block the partial sums over its rows of
// dZ3 (db3), of d_out H3 (dw4), of d_out (db4) and of the loss terms.  Lane l
// of each warp handles columns 8l .. 8l + 7 with 16-byte loads; the 8 warps
// take rows w, w + 8, ... of the block's chunk, two rows per step so that four
// loads are in flight; the warps' sums are added in warp order (deterministic).
constexpr int HB_CHUNKS = 1024;   // most row chunks (blocks) of the head kernel
__device__ __forceinline__ void hb_row(const uint4 &zv, const uint4 &hv, float d, const float (&wv)[8],
                                       float (&s3)[8], float (&s4)[8], uint4 &ov) {
    const __nv_bfloat162 *z2 = reinterpret_cast<const __nv_bfloat162 *>(&zv);
    const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&hv);
    __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&ov);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 z = __bfloat1622float2(z2[k]), h = __bfloat1622float2(h2[k]);
        const __nv_bfloat16 a = __float2bfloat16(d * wv[2 * k] * dsilu(z.x));
        const __nv_bfloat16 b = __float2bfloat16(d * wv[2 * k + 1] * dsilu(z.y));
        o2[k] = __halves2bfloat162(a, b);
        s3[2 * k] += __bfloat162float(a);
        s3[2 * k + 1] += __bfloat162float(b);
        s4[2 * k] = fmaf(d, h.x, s4[2 * k]);
        s4[2 * k + 1] = fmaf(d, h.y, s4[2 * k + 1]);
    }
}
__global__ void __launch_bounds__(256, 3)
    k_head_back_v8(const float *__restrict__ out, const float *__restrict__ y, int64_t rows,
                   int64_t valid, float inv_b, const float *__restrict__ w4, const bf16 *__restrict__ Z3,
                   const bf16 *__restrict__ H3, int width, float *__restrict__ dout, bf16 *__restrict__ dZ3,
                   float *__restrict__ part_db3, float *__restrict__ part_dw4,
                   float *__restrict__ part_db4, float *__restrict__ part_loss) {
    __shared__ float sh[2][8][257];
    __shared__ float shs[2][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(rows, r0 + per);
    const bool act = 8 * lane < width;
    float wv[8], s3[8], s4[8], sd = 0.f, sl = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        wv[k] = act ? w4[8 * lane + k] : 0.f;
        s3[k] = 0.f;
        s4[k] = 0.f;
    }
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t r = r0 + w; r < r1; r += 16) {
        const int64_t rb = r + 8;
        const bool hb = rb < r1;
        const float ea = r < valid ? out[r] - y[r] : 0.f;
        const float eb = hb && rb < valid ? out[rb] - y[rb] : 0.f;
        uint4 za = zero, ha = zero, zb = zero, hbv = zero;
        if (act) {
            za = *reinterpret_cast<const uint4 *>(Z3 + r * width + 8 * lane);
            ha = *reinterpret_cast<const uint4 *>(H3 + r * width + 8 * lane);
            if (hb) {
                zb = *reinterpret_cast<const uint4 *>(Z3 + rb * width + 8 * lane);
                hbv = *reinterpret_cast<const uint4 *>(H3 + rb * width + 8 * lane);
            }
        }
        const float da = ea * inv_b, db = eb * inv_b;
        sd += da + db;
        sl += 0.5f * ea * ea + 0.5f * eb * eb;
        if (lane == 0) {
            dout[r] = da;
            if (hb) dout[rb] = db;
        }
        if (act) {
            uint4 o;
            hb_row(za, ha, da, wv, s3, s4, o);
            *reinterpret_cast<uint4 *>(dZ3 + r * width + 8 * lane) = o;
            if (hb) {
                hb_row(zb, hbv, db, wv, s3, s4, o);
                *reinterpret_cast<uint4 *>(dZ3 + rb * width + 8 * lane) = o;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        sh[0][w][8 * lane + k] = s3[k];
        sh[1][w][8 * lane + k] = s4[k];
    }
    if (lane == 0) {
        shs[0][w] = sd;
        shs[1][w] = sl;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < width; c += blockDim.x) {
        float a = sh[0][0][c], b = sh[1][0][c];
        for (int k = 1; k < 8; ++k) {
            a += sh[0][k][c];
            b += sh[1][k][c];
        }
        part_db3[(int64_t)blockIdx.x * width + c] = a;
        part_dw4[(int64_t)blockIdx.x * width + c] = b;
    }
    if (threadIdx.x < 2) {
        float t = shs[threadIdx.x][0];
        for (int k = 1; k < 8; ++k) t += shs[threadIdx.x][k];
        (threadIdx.x ? part_loss : part_db4)[blockIdx.x] = t;
    }
}

// column sums over rows of a BF16 (or FP32 when F) matrix: out[c] = sum_r X[r][c]
// Column sums over rows, two passes in a fixed order (deterministic):
// part[k][c] = sum of wgt[r] X[r][c] over the rows r of chunk k (wgt null: 1),
// 32 columns x 8 row lanes per block (coalesced along the columns); then
// out[c] = sum_k part[k][c].
constexpr int RED_CHUNKS = 64;
template <typename T>
__global__ void k_colsum_part(const T *__restrict__ X, const float *__restrict__ wgt, int64_t rows, int cols,
                              float *__restrict__ part) {
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cx;
    const int64_t per = (rows + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = (int64_t)blockIdx.y * per, r1 = min(rows, r0 + per);
    float s = 0.f;
    if (c < cols)
        for (int64_t r = r0 + ry; r < r1; r += 8) {
            float x;
            if constexpr (sizeof(T) == 2) x = __bfloat162float(X[r * cols + c]);
            else x = (float)X[r * cols + c];
            s += wgt ? wgt[r] * x : x;
        }
    __shared__ float sh[8][33];
    sh[ry][cx] = s;
    __syncthreads();
    if (ry == 0 && c < cols) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += sh[i][cx];
        part[(int64_t)blockIdx.y * cols + c] = t;
    }
}
// out[c] = sum_k part[k][c] for up to four (part, chunks, cols, out) segments
// (blockIdx.y): 32 columns per block (lane: column), the 32 warps take chunks
// w, w + 32, ... and their sums are added in warp order (deterministic)
struct FinSeg {
    const float *part;
    float *out;
    int chunks, cols;
};
struct FinSegs {
    FinSeg s[4];
};
__global__ void __launch_bounds__(1024) k_colsum_fin(const __grid_constant__ FinSegs segs) {
    __shared__ float sh[32][33];
    const FinSeg &g = segs.s[blockIdx.y];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    if (blockIdx.x * 32 >= g.cols) return;   // uniform over the block
    float t = 0.f;
    if (c < g.cols) {
#pragma unroll 4
        for (int k = w; k < g.chunks; k += 32) t += g.part[(int64_t)k * g.cols + c];
    }
    sh[w][lane] = t;
    __syncthreads();
    if (w == 0 && c < g.cols) {
        float u = sh[0][lane];
        for (int k = 1; k < 32; ++k) u += sh[k][lane];
        g.out[c] = u;
    }
}
inline void colsum_fin(cudaStream_t st, const FinSegs &segs, int nseg) {
    int cmax = 1;
    for (int i = 0; i < nseg; ++i) cmax = std::max(cmax, segs.s[i].cols);
    k_colsum_fin<<<dim3((unsigned)((cmax + 31) / 32), (unsigned)nseg), 1024, 0, st>>>(segs);
}
inline void colsum_fin(cudaStream_t st, const float *part, int chunks, int cols, float *out) {
    FinSegs segs{};
    segs.s[0] = FinSeg{part, out, chunks, cols};
    colsum_fin(st, segs, 1);
}
// BF16 rows of at most 256 columns (a multiple of 8): lane l of every warp
// reads columns 8l .. 8l + 7 of a row in one 16-byte load, so a warp reads
// whole rows; the 8 warps of a block take every 8th row of the block's chunk,
// and their sums are added in warp order (fixed: deterministic).
constexpr int RED_CHUNKS_V = 1024;   // most row chunks (blocks) of k_colsum_v8
__global__ void __launch_bounds__(256)
    k_colsum_v8(const bf16 *__restrict__ X, const float *__restrict__ wgt, int64_t rows, int cols,
                float *__restrict__ part) {
    __shared__ float sh[8][257];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(rows, r0 + per);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (8 * lane < cols)
        for (int64_t r = r0 + w; r < r1; r += 16) {
            // rows r and r + 8 per step: two loads in flight per lane
            const bool hb = r + 8 < r1;
            const uint4 va = *reinterpret_cast<const uint4 *>(X + r * cols + 8 * lane);
            const uint4 vb = hb ? *reinterpret_cast<const uint4 *>(X + (r + 8) * cols + 8 * lane)
                                : make_uint4(0u, 0u, 0u, 0u);
            const float ga = wgt ? wgt[r] : 1.f, gb = hb ? (wgt ? wgt[r + 8] : 1.f) : 0.f;
            const __nv_bfloat162 *ha = reinterpret_cast<const __nv_bfloat162 *>(&va);
            const __nv_bfloat162 *hbp = reinterpret_cast<const __nv_bfloat162 *>(&vb);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(ha[k]);
                s[2 * k] = fmaf(ga, f.x, s[2 * k]);
                s[2 * k + 1] = fmaf(ga, f.y, s[2 * k + 1]);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(hbp[k]);
                s[2 * k] = fmaf(gb, f.x, s[2 * k]);
                s[2 * k + 1] = fmaf(gb, f.y, s[2 * k + 1]);
            }
        }
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[w][8 * lane + k] = s[k];
    __syncthreads();
    for (int c = threadIdx.x; c < cols; c += blockDim.x) {
        float t = sh[0][c];
        for (int k = 1; k < 8; ++k) t += sh[k][c];
        part[(int64_t)blockIdx.x * cols + c] = t;
    }
}

// partial sums buffer of a network of the given width: the column sums' chunks,
// or the head's four partial vectors
inline size_t red_floats(int w) {
    return std::max({(size_t)RED_CHUNKS * w, (size_t)RED_CHUNKS_V * w, (size_t)HB_CHUNKS * (2 * w + 2)});
}

// out[c] = sum_r wgt[r] X[r][c]; part: red_floats(cols) floats
// row chunks of the 256-thread streaming kernels: per_sm blocks per SM, at
// least 64 rows each
inline int stream_chunks(int64_t rows, int sms, int most, int per_sm = 4) {
    return (int)std::min<int64_t>(std::min<int64_t>(most, per_sm * (int64_t)std::max(1, sms)),
                                  std::max<int64_t>(1, rows / 64));
}

template <typename T>
void colsum(cudaStream_t st, const T *X, const float *wgt, int64_t rows, int cols, float *part, float *out,
            int sms) {
    if constexpr (sizeof(T) == 2) {
        if (cols % 8 == 0 && cols <= 256) {
            const int ch = stream_chunks(rows, sms, RED_CHUNKS_V);
            k_colsum_v8<<<(unsigned)ch, 256, 0, st>>>(X, wgt, rows, cols, part);
            colsum_fin(st, part, ch, cols, out);
            return;
        }
    }
    const int ch = (int)std::min<int64_t>(RED_CHUNKS, std::max<int64_t>(1, rows / 256));
    k_colsum_part<T><<<dim3((unsigned)((cols + 31) / 32), (unsigned)ch), 256, 0, st>>>(X, wgt, rows, cols, part);
    colsum_fin(st, part, ch, cols, out);
}

// Adam on the FP32 master parameters (bias-corrected moments)
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of a weight matrix W[rows][cols] (FP32): row-major and transposed
__global__ void k_to_bf16(const float *__restrict__ W, int rows, int cols, bf16 *__restrict__ Wb,
                          bf16 *__restrict__ WbT) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    const int r = (int)(i / cols), c = (int)(i % cols);
    const bf16 v = __float2bfloat16(W[i]);
    Wb[i] = v;
    if (WbT) WbT[(int64_t)c * rows + r] = v;
}

// X0 = BF16 rows of the input, zero-padded from in_dim to in_pad columns (a
// multiple of 8): one thread per row, eight columns per 16-byte store
__global__ void k_input_bf16(const float *__restrict__ x, int64_t rows, int in_dim, int in_pad,
                             bf16 *__restrict__ X0) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float *xr = x + r * in_dim;
    for (int c0 = 0; c0 < in_pad; c0 += 8) {
        uint4 v;
        uint32_t *vp = &v.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = c0 + 2 * k;
            vp[k] = pack_bf16(c < in_dim ? xr[c] : 0.f, c + 1 < in_dim ? xr[c + 1] : 0.f);
        }
        *reinterpret_cast<uint4 *>(X0 + r * in_pad + c0) = v;
    }
}

// C[r][c] = sum_z ws[z][r][c] (the split-K partials, in slice order)
// 256 threads: 32 consecutive outputs x 8 slice groups; warp g sums slices
// g, g + 8, g + 16, ... of its 32 outputs (coalesced 128-byte rows), then the 8
// group sums are added in group order: a fixed order, so the result is
// deterministic, with 8 x the parallelism of one thread per output.
constexpr int SPLIT_GROUPS = 8;
__global__ void __launch_bounds__(32 * SPLIT_GROUPS)
    k_split_sum(const float *__restrict__ ws, int S, int M, int N, int ldc, float *__restrict__ C) {
    __shared__ float sh[SPLIT_GROUPS][33];
    const int cx = threadIdx.x & 31, gz = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + cx;
    const bool ok = i < (int64_t)M * N;
    const int64_t o = ok ? (i / N) * ldc + i % N : 0, zs = (int64_t)M * ldc;
    float v = 0.f;
    if (ok)
        for (int z = gz; z < S; z += SPLIT_GROUPS) v += ws[z * zs + o];
    sh[gz][cx] = v;
    __syncthreads();
    if (gz == 0 && ok) {
        float t = sh[0][cx];
#pragma unroll
        for (int k = 1; k < SPLIT_GROUPS; ++k) t += sh[k][cx];
        C[o] = t;
    }
}

constexpr int SPLIT_MAX = 128;   // split-K slices at most (workspace SPLIT_MAX x M x ldc floats)

// Tensor map of a BF16 operand for the tcgen05 kernel's TMA stage copies,
// 128-byte swizzle, zero fill outside: K-contiguous src[r * ld + k] (rows x K,
// box 64 K x 128 rows) or, transposed, src[k * ld + r] (box 64 rows x 64 K).
// false (the kernel then copies the operand with cp.async) when the driver's
// encoder is unavailable or the operand breaks a TMA rule: base and row
// stride multiples of 16 bytes.
bool t5_tensor_map(CUtensorMap *map, const bf16 *src, int rows, int K, int ld, bool trans) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode || !src || rows < 1 || K < 1 || ld < (trans ? rows : K) ||
        (reinterpret_cast<uintptr_t>(src) & 15) || ((int64_t)ld * 2) % 16)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(trans ? rows : K), (cuuint64_t)(trans ? K : rows)};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64, trans ? 64u : 128u}, estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(src), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of a BF16 (or FP32) matrix src[r * ld + c] (rows x cols) with
// boxes of 128 bytes of columns (64 BF16, 32 FP32) x box_rows rows in the
// 128-byte swizzle (TMA loads and stores of the persistent kernel); false when
// the encoder is unavailable or a TMA rule is broken (base and row stride
// multiples of 16 bytes, box_rows <= 256).
bool t6_tensor_map(CUtensorMap *map, const void *src, int rows, int cols, int ld, int box_rows,
                   bool f32 = false) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    const int es = f32 ? 4 : 2;   // element bytes; a box row is 128 bytes either way
    if (!encode || !src || rows < 1 || cols < 1 || ld < cols || box_rows < 1 || box_rows > 256 ||
        (reinterpret_cast<uintptr_t>(src) & 15) || ((int64_t)ld * es) % 16)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows}, estr[2] = {1, 1};
    return encode(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void *>(src), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// kind 0: tcgen05 kernel with TMA operand copies where the operand allows them,
// 2: the same kernel with cp.async copies only, 1: warp-level mma.sync kernel
// (same operands, epilogues).
// A plain-FP32 GEMM with a long K and few output tiles (the weight gradients,
// K = rows) is split along K over about two CTAs per SM, its partials summed
// by k_split_sum in a fixed order (ws: SPLIT_MAX x M x ldc floats).
template <bool AT, bool BT, int EPI>
void gemm(cudaStream_t st, int kind, int *flags, float *ws, int sms, int M, int N, int K, const bf16 *A,
          int lda, const bf16 *B, int ldb, float *C, int ldc, const float *bias, bf16 *H, int ldh,
          bf16 *Z, int ldz) {
    const int tiles = ((M + 127) / 128) * ((N + 127) / 128);
    int S = 1;
    if (EPI == EPI_F32 && ws) S = std::max(1, std::min({K / 512, 2 * sms / std::max(1, tiles), SPLIT_MAX}));
    const int kslice = S > 1 ? (K + S - 1) / S / 64 * 64 + 64 : K;
    if (S > 1) S = (K + kslice - 1) / kslice;
    float *Cw = S > 1 ? ws : C;
    // the persistent warp-specialised kernel: the BF16 epilogues with K-contiguous
    // operands and the FP32 weight gradients with MN-contiguous ones, N <= 256 a
    // multiple of 32, when every operand allows TMA; the same K slices as the
    // kernels below, so every form sums the same partials in the same order
    const bool t6_shape = EPI == EPI_F32 ? (AT && BT && M % 32 == 0 && (S == 1 || kslice % 64 == 0))
                                         : (!AT && !BT && (EPI != EPI_DSILU || ldz % 8 == 0));
    if (kind == 0 && t6_shape && N % 32 == 0 && N <= 256) {
        CUtensorMap ma, mb, mh, mz;
        memset(&mh, 0, sizeof(mh));
        memset(&mz, 0, sizeof(mz));
        // boxes: K-contiguous A 64 x 128 rows, B 64 x N rows; MN-contiguous 64 x 64
        bool t6 = AT ? t6_tensor_map(&ma, A, K, M, lda, 64) : t6_tensor_map(&ma, A, M, K, lda, 128);
        if (t6) t6 = BT ? t6_tensor_map(&mb, B, K, N, ldb, 64) : t6_tensor_map(&mb, B, N, K, ldb, N);
        if (t6 && EPI != EPI_F32)
            t6 = t6_tensor_map(&mh, H, M, N, ldh, 32) &&
                 t6_tensor_map(&mz, Z, M, N, ldz, 32);   // Z stored (forward) or loaded (x SiLU'(Z))
        if (t6 && EPI == EPI_F32)   // the FP32 results: S slices of M rows, boxes 32 x 32
            t6 = t6_tensor_map(&mh, Cw, S * M, N, ldc, 32, true);
        if (t6) {
            static bool attr6 = false;   // 225 KB of dynamic shared memory, set once per instance
            if (!attr6) {
                cudaFuncSetAttribute((const void *)k_gemm_t6<AT, BT, EPI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, T6_SMEM);
                attr6 = true;
            }
            const int mblocks = (M + 127) / 128, tiles6 = mblocks * S;
            k_gemm_t6<AT, BT, EPI><<<std::max(1, std::min(tiles6, sms)), T6_THREADS, T6_SMEM, st>>>(
                M, N, K, kslice, mblocks, Cw, ldc, bias, flags, ma, mb, mh, mz);
            if (S > 1)
                k_split_sum<<<(unsigned)(((int64_t)M * N + 31) / 32), 32 * SPLIT_GROUPS, 0, st>>>(ws, S, M, N, ldc, C);
            return;
        }
    }
    if (kind == 0 || kind == 2) {
        static bool attr = false;   // 69 KB of dynamic shared memory, set once per instance
        if (!attr) {
            cudaFuncSetAttribute((const void *)k_gemm_t5<AT, BT, EPI>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, T5_SMEM);
            attr = true;
        }
        // TMA operand copies: a box (64 K) never crosses a K slice's end, since
        // slices start and end on multiples of 64 or at K, where zero fill begins
        CUtensorMap ma, mb, mh, mz;
        memset(&ma, 0, sizeof(ma));
        memset(&mb, 0, sizeof(mb));
        memset(&mh, 0, sizeof(mh));
        memset(&mz, 0, sizeof(mz));
        int tma = 0;
        if (kind == 0 && (S == 1 || kslice % T5_K == 0)) {
            if (t5_tensor_map(&ma, A, M, K, lda, AT)) tma |= 1;
            if (t5_tensor_map(&mb, B, N, K, ldb, BT)) tma |= 2;
        }
        // BF16 outputs by TMA stores (boxes of 64 columns x 128 rows); the
        // x SiLU'(Z) epilogue reads Z rows in 16-byte pieces: N and ldz multiples of 8
        if (kind == 0 && EPI != EPI_F32 && N % 8 == 0 && (EPI != EPI_DSILU || ldz % 8 == 0)) {
            if (t5_tensor_map(&mh, H, M, N, ldh, false)) tma |= 4;
            if (EPI == EPI_BIAS_SILU && t5_tensor_map(&mz, Z, M, N, ldz, false)) tma |= 8;
        }
        dim3 grid((N + T5_N - 1) / T5_N, (M + T5_M - 1) / T5_M, S);
        k_gemm_t5<AT, BT, EPI><<<grid, T5_THREADS, T5_SMEM, st>>>(M, N, K, kslice, A, lda, B, ldb, Cw, ldc,
                                                                   bias, H, ldh, Z, ldz, flags, ma, mb, mh, mz,
                                                                   tma);
    } else {
        dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM, S);
        k_gemm_bf16<AT, BT, EPI><<<grid, G_THREADS, 0, st>>>(M, N, K, kslice, A, lda, B, ldb, Cw, ldc, bias,
                                                             H, ldh, Z, ldz);
    }
    if (S > 1)
        k_split_sum<<<(unsigned)(((int64_t)M * N + 31) / 32), 32 * SPLIT_GROUPS, 0, st>>>(ws, S, M, N, ldc, C);
}

uint64_t mix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace rsot

using rsot::bf16;

struct rsot_mlp {
    int in_dim = 0, in_pad = 0, width = 0;
    int64_t cap = 0;   // rows of the activation buffers
    cudaStream_t stream = nullptr;
    // parameter block (FP32): W1 [w][in_pad], b1 [w], W2 [w][w], b2, W3 [w][w], b3, w4 [w], b4 [1]
    int64_t off[8] = {0}, n_params = 0;
    float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
    int64_t step = 0;
    bf16 *W1b = nullptr, *W1bT = nullptr, *W2b = nullptr, *W2bT = nullptr, *W3b = nullptr, *W3bT = nullptr;
    // activations
    bf16 *X0 = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *dZ = nullptr, *dZ2 = nullptr;
    bf16 *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr;   // pre-activations, rounded to BF16
    float *dH = nullptr, *out = nullptr, *dout = nullptr,
          *lt = nullptr, *xin = nullptr, *yin = nullptr, *scal = nullptr;
    int gemm_kind = 0;       // 0: tcgen05 GEMM (TMA), 1: mma.sync GEMM, 2: tcgen05 GEMM (cp.async)
    float *ws = nullptr;     // split-K partials of the weight-gradient GEMMs
    float *red = nullptr;    // partials of the column sums (RED_CHUNKS x width)
    int sms = 1;
    int *flags = nullptr;    // device error flags of the GEMM kernels (kErrTimeout)
};

namespace rsot {
namespace {

cudaError_t mlp_refresh_bf16(rsot_mlp *m) {
    const int w = m->width;
    cudaStream_t st = m->stream;
    k_to_bf16<<<(w * m->in_pad + 255) / 256, 256, 0, st>>>(m->P + m->off[0], w, m->in_pad, m->W1b, m->W1bT);
    k_to_bf16<<<(w * w + 255) / 256, 256, 0, st>>>(m->P + m->off[2], w, w, m->W2b, m->W2bT);
    k_to_bf16<<<(w * w + 255) / 256, 256, 0, st>>>(m->P + m->off[4], w, w, m->W3b, m->W3bT);
    return cudaGetLastError();
}

cudaError_t mlp_reserve(rsot_mlp *m, int64_t rows) {
    if (rows <= m->cap) return cudaSuccess;
    const int64_t r = (rows + 127) / 128 * 128;
    void *ptrs[] = {m->X0, m->H1, m->H2, m->H3, m->dZ, m->dZ2, m->Z1, m->Z2, m->Z3, m->dH,
                    m->out, m->dout, m->lt, m->xin, m->yin};
    for (void *q : ptrs) cudaFree(q);
    const int w = m->width;
    cudaError_t e = cudaSuccess;
#define MA(ptr, cnt) \
    if (!e) e = cudaMalloc(&(ptr), (size_t)(cnt) * sizeof(*(ptr)))
    MA(m->X0, r * m->in_pad);
    MA(m->H1, r * w);
    MA(m->H2, r * w);
    MA(m->H3, r * w);
    MA(m->dZ, r * w);
    MA(m->dZ2, r * w);
    MA(m->Z1, r * w);
    MA(m->Z2, r * w);
    MA(m->Z3, r * w);
    MA(m->dH, r * w);
    MA(m->out, r);
    MA(m->dout, r);
    MA(m->lt, r);
    MA(m->xin, r * m->in_dim);
    MA(m->yin, r);
#undef MA
    if (!e) {
        m->cap = r;
        cudaMemset(m->X0, 0, r * m->in_pad * sizeof(bf16));
        cudaMemset(m->xin, 0, r * m->in_dim * sizeof(float));
        cudaMemset(m->yin, 0, r * sizeof(float));
    }
    return e;
}

// a GEMM wait that gave up (flag read with the call's results): cleared, reported
rsot_status mlp_take_flags(rsot_mlp *m, int fl) {
    if (!fl) return RSOT_OK;
    cudaMemset(m->flags, 0, sizeof(int));
    return RSOT_ERR_TIMEOUT;
}

// forward on rows (padded to 128) from m->xin; result in m->out
void mlp_forward(rsot_mlp *m, int64_t rows) {
    const int w = m->width, R = (int)((rows + 127) / 128 * 128);
    cudaStream_t st = m->stream;
    k_input_bf16<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(m->xin, R, m->in_dim,
                                                                                 m->in_pad, m->X0);
    gemm<false, false, EPI_BIAS_SILU>(st, m->gemm_kind, m->flags, m->ws, m->sms, R, w, m->in_pad, m->X0, m->in_pad, m->W1b, m->in_pad, nullptr,
                                      w, m->P + m->off[1], m->H1, w, m->Z1, w);
    gemm<false, false, EPI_BIAS_SILU>(st, m->gemm_kind, m->flags, m->ws, m->sms, R, w, w, m->H1, w, m->W2b, w, nullptr, w, m->P + m->off[3],
                                      m->H2, w, m->Z2, w);
    gemm<false, false, EPI_BIAS_SILU>(st, m->gemm_kind, m->flags, m->ws, m->sms, R, w, w, m->H2, w, m->W3b, w, nullptr, w, m->P + m->off[5],
                                      m->H3, w, m->Z3, w);
    if (w % 8 == 0 && w <= 256)
        k_head_v8<<<(unsigned)((R + 7) / 8), 256, 0, st>>>(m->H3, w, R, m->P + m->off[6], m->P + m->off[7], m->out);
    else
        k_head<<<(unsigned)((R + 7) / 8), 256, 0, st>>>(m->H3, w, R, m->P + m->off[6], m->P + m->off[7], m->out);
}

// forward + backward: gradients of loss = sum_valid (out - y)^2 / (2 rows) into m->G;
// loss_sum (device, one float) receives the sum of the loss terms 0.5 (out - y)^2
void mlp_backward(rsot_mlp *m, int64_t rows, float *loss_sum) {
    const int w = m->width, R = (int)((rows + 127) / 128 * 128);
    cudaStream_t st = m->stream;
    mlp_forward(m, rows);
    float *G = m->G;
    if (w % 8 == 0 && w <= 256) {
        // head back-propagation with its column sums: dw4 = sum_r dout_r H3[r],
        // db3 = colsum dZ3, db4 = sum_r dout_r and the loss
        const int ch = stream_chunks(R, m->sms, HB_CHUNKS, 3);   // one wave of three blocks per SM
        float *p3 = m->red, *p4 = p3 + (size_t)HB_CHUNKS * w, *p5 = p4 + (size_t)HB_CHUNKS * w,
              *p6 = p5 + HB_CHUNKS;
        k_head_back_v8<<<(unsigned)ch, 256, 0, st>>>(m->out, m->yin, R, rows, 1.0f / (float)rows,
                                                     m->P + m->off[6], m->Z3, m->H3, w, m->dout, m->dZ,
                                                     p3, p4, p5, p6);
        FinSegs segs{};
        segs.s[0] = FinSeg{p4, G + m->off[6], ch, w};
        segs.s[1] = FinSeg{p3, G + m->off[5], ch, w};
        segs.s[2] = FinSeg{p5, G + m->off[7], ch, 1};
        segs.s[3] = FinSeg{p6, loss_sum, ch, 1};
        colsum_fin(st, segs, loss_sum ? 4 : 3);
    } else {
        k_head_back<<<(unsigned)((R + 7) / 8), 256, 0, st>>>(m->out, m->yin, R, rows, 1.0f / (float)rows,
                                                             m->P + m->off[6], m->Z3, w, m->dout, m->dZ, m->lt);
        colsum<bf16>(st, m->H3, m->dout, R, w, m->red, G + m->off[6], m->sms);   // dw4 = sum_r dout_r H3[r]
        colsum<float>(st, m->dout, nullptr, R, 1, m->red, G + m->off[7], m->sms);
        colsum<bf16>(st, m->dZ, nullptr, R, w, m->red, G + m->off[5], m->sms);   // db3 = colsum dZ3
        if (loss_sum) colsum<float>(st, m->lt, nullptr, R, 1, m->red, loss_sum, m->sms);
    }
    // layer 3: dW3 = dZ3^T H2, dZ2 = (dZ3 W3) * SiLU'(Z2)
    gemm<true, true, EPI_F32>(st, m->gemm_kind, m->flags, m->ws, m->sms, w, w, R, m->dZ, w, m->H2, w, G + m->off[4], w, nullptr, nullptr, 0, nullptr, 0);
    gemm<false, false, EPI_DSILU>(st, m->gemm_kind, m->flags, m->ws, m->sms, R, w, w, m->dZ, w, m->W3bT, w, nullptr, 0, nullptr, m->dZ2, w, m->Z2, w);
    // layer 2
    gemm<true, true, EPI_F32>(st, m->gemm_kind, m->flags, m->ws, m->sms, w, w, R, m->dZ2, w, m->H1, w, G + m->off[2], w, nullptr, nullptr, 0, nullptr, 0);
    colsum<bf16>(st, m->dZ2, nullptr, R, w, m->red, G + m->off[3], m->sms);
    gemm<false, false, EPI_DSILU>(st, m->gemm_kind, m->flags, m->ws, m->sms, R, w, w, m->dZ2, w, m->W2bT, w, nullptr, 0, nullptr, m->dZ, w, m->Z1, w);
    // layer 1: dW1 = dZ1^T X0, db1 = colsum dZ1
    gemm<true, true, EPI_F32>(st, m->gemm_kind, m->flags, m->ws, m->sms, w, m->in_pad, R, m->dZ, w, m->X0, m->in_pad, G + m->off[0], m->in_pad,
                              nullptr, nullptr, 0, nullptr, 0);
    colsum<bf16>(st, m->dZ, nullptr, R, w, m->red, G + m->off[1], m->sms);
}

}  // namespace
}  // namespace rsot

using namespace rsot;

extern "C" {

void rsot_mlp_destroy(rsot_mlp *m) {
    if (!m) return;
    void *ptrs[] = {m->P, m->G, m->Mo, m->Vo, m->W1b, m->W1bT, m->W2b, m->W2bT, m->W3b, m->W3bT,
                    m->X0, m->H1, m->H2, m->H3, m->dZ, m->dZ2, m->Z1, m->Z2, m->Z3, m->dH, m->out,
                    m->dout, m->lt, m->xin, m->yin, m->scal, m->flags, m->ws, m->red};
    for (void *q : ptrs) cudaFree(q);
    delete m;
}

rsot_status rsot_mlp_create(int in_dim, int width, uint64_t seed, rsot_mlp **out) {
    if (!out || in_dim < 1 || in_dim > 64 || width < 8 || width > 1024 || width % 8) return RSOT_ERR_ARG;
    rsot_mlp *m = new rsot_mlp();
    m->in_dim = in_dim;
    m->in_pad = (in_dim + 31) / 32 * 32;
    m->width = width;
    const int w = width;
    const int64_t sizes[8] = {(int64_t)w * m->in_pad, w, (int64_t)w * w, w, (int64_t)w * w, w, w, 1};
    for (int i = 0; i < 8; ++i) {
        m->off[i] = m->n_params;
        m->n_params += sizes[i];
    }
    // initialisation: uniform(-a, a), a = sqrt(6 / fan_in) for the hidden layers (SiLU),
    // sqrt(3 / fan_in) for the head; zero biases; padded input columns zero
    std::vector<float> h(m->n_params, 0.f);
    uint64_t s = seed;
    auto uni = [&](double a) { return (float)(a * (2.0 * ((mix64(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.0)); };
    for (int r = 0; r < w; ++r)
        for (int c = 0; c < in_dim; ++c) h[m->off[0] + (int64_t)r * m->in_pad + c] = uni(sqrt(6.0 / in_dim));
    for (int64_t i = 0; i < (int64_t)w * w; ++i) h[m->off[2] + i] = uni(sqrt(6.0 / w));
    for (int64_t i = 0; i < (int64_t)w * w; ++i) h[m->off[4] + i] = uni(sqrt(6.0 / w));
    for (int i = 0; i < w; ++i) h[m->off[6] + i] = uni(sqrt(3.0 / w));
    cudaError_t e = cudaSuccess;
    if (!e) e = cudaMalloc(&m->P, m->n_params * 4);
    if (!e) e = cudaMalloc(&m->G, m->n_params * 4);
    if (!e) e = cudaMalloc(&m->Mo, m->n_params * 4);
    if (!e) e = cudaMalloc(&m->Vo, m->n_params * 4);
    if (!e) e = cudaMalloc(&m->W1b, (size_t)w * m->in_pad * 2);
    if (!e) e = cudaMalloc(&m->W1bT, (size_t)w * m->in_pad * 2);
    if (!e) e = cudaMalloc(&m->W2b, (size_t)w * w * 2);
    if (!e) e = cudaMalloc(&m->W2bT, (size_t)w * w * 2);
    if (!e) e = cudaMalloc(&m->W3b, (size_t)w * w * 2);
    if (!e) e = cudaMalloc(&m->W3bT, (size_t)w * w * 2);
    if (!e) e = cudaMalloc(&m->scal, 16);
    if (!e) e = cudaMalloc(&m->flags, sizeof(int));
    if (!e) e = cudaMalloc(&m->ws, (size_t)SPLIT_MAX * w * std::max(w, m->in_pad) * sizeof(float));
    if (!e) e = cudaMalloc(&m->red, red_floats(w) * sizeof(float));
    int dev = 0;
    if (!e) e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaMemset(m->flags, 0, sizeof(int));
    if (!e) e = cudaMemcpy(m->P, h.data(), m->n_params * 4, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(m->Mo, 0, m->n_params * 4);
    if (!e) e = cudaMemset(m->Vo, 0, m->n_params * 4);
    if (!e) e = cudaMemset(m->G, 0, m->n_params * 4);
    if (!e) e = mlp_refresh_bf16(m);
    if (!e) e = cudaStreamSynchronize(m->stream);
    if (e) {
        cudaGetLastError();
        rsot_mlp_destroy(m);
        return RSOT_ERR_CUDA;
    }
    *out = m;
    return RSOT_OK;
}

int64_t rsot_mlp_num_params(const rsot_mlp *m) { return m ? m->n_params : 0; }

rsot_status rsot_mlp_set_gemm_kernel(rsot_mlp *m, int kind) {
    if (!m || kind < 0 || kind > 2) return RSOT_ERR_ARG;
    m->gemm_kind = kind;
    return RSOT_OK;
}

rsot_status rsot_mlp_set_stream(rsot_mlp *m, void *stream) {
    if (!m) return RSOT_ERR_ARG;
    m->stream = (cudaStream_t)stream;
    return RSOT_OK;
}

rsot_status rsot_mlp_get_params(rsot_mlp *m, float *out) {
    if (!m || !out) return RSOT_ERR_ARG;
    return cudaMemcpy(out, m->P, m->n_params * 4, cudaMemcpyDefault) ? RSOT_ERR_CUDA : RSOT_OK;
}

rsot_status rsot_mlp_set_params(rsot_mlp *m, const float *in) {
    if (!m || !in) return RSOT_ERR_ARG;
    if (cudaMemcpy(m->P, in, m->n_params * 4, cudaMemcpyDefault)) return RSOT_ERR_CUDA;
    mlp_refresh_bf16(m);
    return cudaStreamSynchronize(m->stream) ? RSOT_ERR_CUDA : RSOT_OK;
}

rsot_status rsot_mlp_forward(rsot_mlp *m, int64_t rows, const float *x, float *y_out) {
    if (!m || rows < 1 || !x || !y_out) return RSOT_ERR_ARG;
    cudaError_t e = mlp_reserve(m, rows);
    if (!e) e = cudaMemcpyAsync(m->xin, x, (size_t)rows * m->in_dim * 4, cudaMemcpyDefault, m->stream);
    if (!e) {
        mlp_forward(m, rows);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(y_out, m->out, (size_t)rows * 4, cudaMemcpyDefault, m->stream);
    int fl = 0;
    if (!e) e = cudaMemcpyAsync(&fl, m->flags, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    if (!e) e = cudaStreamSynchronize(m->stream);
    if (e) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    return mlp_take_flags(m, fl);
}

rsot_status rsot_mlp_gradients(rsot_mlp *m, int64_t rows, const float *x, const float *y,
                               float *loss_out, float *grad_out) {
    if (!m || rows < 1 || !x || !y) return RSOT_ERR_ARG;
    cudaError_t e = mlp_reserve(m, rows);
    const int64_t R = (rows + 127) / 128 * 128;
    // the padding rows (rows .. R) are zeroed; the copies fill the others
    if (!e && R > rows) e = cudaMemsetAsync(m->xin + rows * m->in_dim, 0, (size_t)(R - rows) * m->in_dim * 4, m->stream);
    if (!e && R > rows) e = cudaMemsetAsync(m->yin + rows, 0, (size_t)(R - rows) * 4, m->stream);
    if (!e) e = cudaMemcpyAsync(m->xin, x, (size_t)rows * m->in_dim * 4, cudaMemcpyDefault, m->stream);
    if (!e) e = cudaMemcpyAsync(m->yin, y, (size_t)rows * 4, cudaMemcpyDefault, m->stream);
    if (!e) {
        mlp_backward(m, rows, m->scal);
        e = cudaGetLastError();
    }
    float l = 0.f;
    if (!e) e = cudaMemcpyAsync(&l, m->scal, 4, cudaMemcpyDeviceToHost, m->stream);
    if (!e && grad_out) e = cudaMemcpyAsync(grad_out, m->G, m->n_params * 4, cudaMemcpyDefault, m->stream);
    int fl = 0;
    if (!e) e = cudaMemcpyAsync(&fl, m->flags, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    if (!e) e = cudaStreamSynchronize(m->stream);
    if (e) {
        cudaGetLastError();
        return RSOT_ERR_CUDA;
    }
    const rsot_status fs = mlp_take_flags(m, fl);
    if (fs) return fs;
    if (loss_out) *loss_out = l / (float)rows;
    return RSOT_OK;
}

rsot_status rsot_mlp_train_step(rsot_mlp *m, int64_t rows, const float *x, const float *y, float lr,
                                float *loss_out) {
    rsot_status s = rsot_mlp_gradients(m, rows, x, y, loss_out, nullptr);
    if (s) return s;
    ++m->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    k_adam<<<(unsigned)((m->n_params + 255) / 256), 256, 0, m->stream>>>(m->P, m->G, m->Mo, m->Vo,
                                                                        m->n_params, lr, b1, b2, 1e-8f,
                                                                        c1, c2);
    cudaError_t e = mlp_refresh_bf16(m);
    if (!e) e = cudaStreamSynchronize(m->stream);
    return e ? (cudaGetLastError(), RSOT_ERR_CUDA) : RSOT_OK;
}

}  // extern "C"
