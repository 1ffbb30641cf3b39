// mlp_gemm.cu -- the training GEMM of the initial-guess network on the
// 5th-generation tensor cores (tcgen05, TMEM accumulators): an extension, the
// paper has no counterpart.
//
// C[M x N] = epi(op(A)[M x K] op(B)[K x N]) with FP32 operands in global
// memory, rounded to BF16 when they are staged into shared memory (the
// rounding points of the network's BF16 arithmetic), FP32 accumulation in
// TMEM.  One CTA (256 threads) computes a 128 x BN tile, BN = N rounded up to
// a multiple of 16 (at most 256), and walks K in chunks of 64 through two
// shared-memory stages:
//
//   all threads    load the chunk's A rows and B columns (FP32, either
//                  layout), round them to BF16 and store them in the K-major
//                  canonical layout of the UMMA descriptors (8-row x 16-byte
//                  core matrices);
//   thread 0       issues 4 tcgen05.mma (M = 128, N = BN, K = 16) and commits
//                  them to the stage's mbarrier, while the other threads go on
//                  staging the next chunk into the other stage;
//   epilogue       warp w reads TMEM lanes 32 (w % 4) .. (its tile rows) and
//                  every other group of 8 columns (w / 4 picks which), adds
//                  the bias, applies ReLU (keeping the pre-activation) or the
//                  ReLU mask of the backward pass, and stores FP32.
//
// Weight gradients (K = batch, M and N <= 256) split K over up to 32 CTAs;
// each writes its partial tile to a workspace that a second kernel sums in a
// fixed order, so results are deterministic.  Every mbarrier wait is bounded:
// one that runs out raises the error flag, the CTA waits (bounded) for its own
// MMAs and frees its TMEM.
#include <atomic>

#include "fsi_internal.cuh"
#include "tc_common.cuh"

namespace fsi {
namespace {

using namespace tc;

constexpr int TM = 128;       // tile rows (MMA M)
constexpr int BK = 64;        // K per stage (4 MMAs of K = 16)
constexpr int KCH = BK / 8;   // 16-byte chunks along K in a stage
constexpr int kThreads = 256;
constexpr uint32_t SZ_A = TM * BK * 2;      // 16 KB
constexpr uint32_t SZ_B = 256 * BK * 2;     // 32 KB (BN <= 256)
constexpr uint32_t SZ_STAGE = SZ_A + SZ_B;
constexpr uint32_t SMEM_BYTES = 2 * SZ_STAGE;  // 96 KB
constexpr int kMaxSplit = 32;

__global__ void __launch_bounds__(kThreads) tc_gemm_kernel(const TcGemm g, float *work, int *err)
{
    extern __shared__ __align__(128) uint8_t sm[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * g.BN;
    const uint32_t s0 = smem_u32(sm);
    const uint32_t bar[2] = {smem_u32(&bars[0]), smem_u32(&bars[1])};
    // K range of this CTA (split K: blockIdx.z of gridDim.z slices of whole chunks)
    const int nchunks_all = (g.K + BK - 1) / BK;
    const int per = (nchunks_all + gridDim.z - 1) / gridDim.z;
    const int c_begin = blockIdx.z * per;
    const int c_end = min(nchunks_all, c_begin + per);
    const int nch = max(0, c_end - c_begin);
    // TMEM columns: a power of two >= 32 holding BN FP32 columns
    uint32_t cols = 32;
    while ((int)cols < g.BN) cols <<= 1;

    if (tid == 0) {
        abort_flag = 0;
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_holder), cols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_holder;
    const uint32_t idesc = idesc_bf16(TM, g.BN);
    // parity of the commit issued on each stage and not yet observed (-1: none)
    int pending[2] = {-1, -1};

    for (int c = 0; c < nch && !abort_flag; ++c) {
        const int st = c & 1;
        const int k0 = (c_begin + c) * BK;
        uint8_t *sa = sm + st * SZ_STAGE;
        uint8_t *sb = sa + SZ_A;
        // the MMAs of chunk c - 2 read this stage: wait for them
        if (c >= 2) {
            const bool ok = mbar_wait(bar[st], ((c - 2) >> 1) & 1);
            if (ok) pending[st] = -1;
            else atomicExch(&abort_flag, 1);
            __syncthreads();
            if (abort_flag) break;
        }
        // stage A: TM rows x BK, one (row, 8-element chunk) per task
        for (int t = tid; t < TM * KCH; t += kThreads) {
            int r, q;
            if (g.transA) { r = t % TM; q = t / TM; }   // rows fastest: coalesced over m
            else { q = t % KCH; r = t / KCH; }          // chunks fastest: coalesced over k
            const int gi = m0 + r, gk = k0 + 8 * q;
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = gk + j;
                v[j] = (gi < g.M && k < g.K)
                           ? (g.transA ? g.A[(int64_t)k * g.lda + gi] : g.A[(int64_t)gi * g.lda + k])
                           : 0.f;
            }
            *reinterpret_cast<uint4 *>(sa + kmaj(r, 8 * q, KCH)) =
                make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                           pack_bf16(v[6], v[7]));
        }
        // stage B^T: BN rows (output columns) x BK
        for (int t = tid; t < g.BN * KCH; t += kThreads) {
            int r, q;
            if (g.transB) { q = t % KCH; r = t / KCH; }  // B stored [N][K]: k contiguous
            else { r = t % g.BN; q = t / g.BN; }         // B stored [K][N]: n contiguous
            const int gj = n0 + r, gk = k0 + 8 * q;
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = gk + j;
                v[j] = (gj < g.N && k < g.K)
                           ? (g.transB ? g.B[(int64_t)gj * g.ldb + k] : g.B[(int64_t)k * g.ldb + gj])
                           : 0.f;
            }
            *reinterpret_cast<uint4 *>(sb + kmaj(r, 8 * q, KCH)) =
                make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                           pack_bf16(v[6], v[7]));
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const uint32_t a0 = s0 + st * SZ_STAGE, b0 = a0 + SZ_A;
#pragma unroll
            for (uint32_t ks = 0; ks < BK / 16; ++ks)
                mma_bf16(tmem, sdesc(a0 + ks * 256, 128, KCH * 128),
                         sdesc(b0 + ks * 256, 128, KCH * 128), idesc, (c > 0 || ks > 0) ? 1u : 0u);
            mma_commit(bar[st]);
        }
        pending[st] = (c >> 1) & 1;
    }
    // all MMAs done: the last commit covers every earlier one
    if (nch > 0 && !abort_flag) {
        const int last = nch - 1;
        const bool ok = mbar_wait(bar[last & 1], (last >> 1) & 1);
        if (ok) pending[0] = pending[1] = -1;
        else atomicExch(&abort_flag, 1);
    }
    __syncthreads();
    fence_after();
    if (!abort_flag) {
        // epilogue: rows 32 (warp % 4) + lane, column groups of 8 split by warp / 4
        const int row = 32 * (warp & 3) + (tid & 31);
        const int gi = m0 + row;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        for (int c8 = warp >> 2; c8 * 8 < g.BN; c8 += 2) {
            float v[8];
            if (nch > 0) tmem_ld8(tmem + lane_base + 8 * c8, v);
            else
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = 0.f;
            if (gi >= g.M) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int gj = n0 + 8 * c8 + j;
                if (gj >= g.N) continue;
                float x = v[j];
                if (gridDim.z > 1) {  // partial sum of a K slice
                    work[((int64_t)blockIdx.z * g.M + gi) * g.N + gj] = x;
                    continue;
                }
                const int64_t o = (int64_t)gi * g.ldc + gj;
                if (g.epi == TC_EPI_BIAS || g.epi == TC_EPI_BIAS_RELU) x += g.bias[gj];
                if (g.epi == TC_EPI_BIAS_RELU) {
                    if (g.Cpre) g.Cpre[o] = x;
                    x = x > 0.f ? x : 0.f;
                }
                if (g.epi == TC_EPI_MASK) x = g.mask[o] > 0.f ? x : 0.f;
                g.C[o] = x;
            }
        }
    }
    if (abort_flag) {
        if (tid == 0) atomicExch(err, 1);
        // nothing may still be in flight when the TMEM is freed
        for (int q = 0; q < 2; ++q)
            if (pending[q] >= 0) mbar_wait(bar[q], (uint32_t)pending[q]);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tmem_free(tmem, cols);
    }
}

// C = sum over the K slices of the partial tiles, in slice order (store epilogue)
__global__ void tc_gemm_reduce_kernel(int M, int N, int splits, const float *work, float *C,
                                      int64_t ldc)
{
    const int64_t total = (int64_t)M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += work[(int64_t)z * total + e];
        C[(e / N) * ldc + e % N] = s;
    }
}

}  // namespace

size_t tc_gemm_work_floats() { return (size_t)kMaxSplit * 256 * 256; }

fsi_status tc_gemm(cudaStream_t s, const TcGemm &g_in, float *work, int *err)
{
    TcGemm g = g_in;
    if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.N > 256)
        return set_error(FSI_ERR_ARG, "tensor-core GEMM: bad shape %d x %d x %d", g.M, g.N, g.K);
    g.BN = (g.N + 15) / 16 * 16;
    static std::atomic<bool> attr_set[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
        FSI_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      SMEM_BYTES),
                 "cudaFuncSetAttribute");
        if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_release);
    }
    const int mt = (g.M + TM - 1) / TM, nt = (g.N + g.BN - 1) / g.BN;
    const int nchunks = (g.K + BK - 1) / BK;
    // split K when the tile grid alone leaves most SMs idle and K is long
    int splits = 1;
    if (g.epi == TC_EPI_STORE && work && mt * nt < sm_count() / 2 && nchunks >= 8) {
        splits = nchunks / 4;
        if (splits > kMaxSplit) splits = kMaxSplit;
        if ((size_t)splits * g.M * g.N > tc_gemm_work_floats()) splits = 1;
        // every slice gets whole chunks, and none is empty
        const int per = (nchunks + splits - 1) / splits;
        splits = (nchunks + per - 1) / per;
    }
    dim3 grid(nt, mt, splits);
    tc_gemm_kernel<<<grid, kThreads, SMEM_BYTES, s>>>(g, work, err);
    FSI_TRY(check_launch("tensor-core gemm"));
    if (splits > 1) {
        const int64_t total = (int64_t)g.M * g.N;
        int blocks = (int)((total + 255) / 256);
        if (blocks > sm_count() * 8) blocks = sm_count() * 8;
        tc_gemm_reduce_kernel<<<blocks, 256, 0, s>>>(g.M, g.N, splits, work, g.C, g.ldc);
        FSI_TRY(check_launch("tensor-core gemm reduce"));
    }
    return FSI_OK;
}

}  // namespace fsi
