// mlp_tc.cu -- fused inference of the initial-guess network on the 5th-
// generation tensor cores (tcgen05, TMEM accumulators).
//
// One persistent CTA per SM (512 threads = four warpgroups, ~223 KB shared
// memory) processes tiles of 128 nodes.  Node row r of the tile is TMEM lane
// r of the accumulators; thread t takes row t % 128, and its warpgroup
// t / 128 takes a quarter of every per-row phase (feature chunks, H1
// columns, layer-3 columns), so that each SMSP has four warps to switch
// between.  Per tile:
//
//   features   the 112 features of each node (27-node stencil of V_n
//              velocity and y_n pressure, the extrapolant 2 d1 - d2),
//              normalised and rounded to BF16, into the A tile X [128 x 112];
//   layer 1    D1 [128 x 256] (TMEM columns 0..255) = X W1^T: 7 MMAs of
//              M=128, N=256, K=16 (kind::f16, BF16 in, FP32 accumulate);
//   layer 2    H1 = BF16(ReLU(D1 + b1)) is written back to shared memory in
//              two K-halves of 128 (the half buffer aliases X), each followed
//              by 8 MMAs accumulating D2 (columns 256..511) = H1 W2^T; the
//              second half is loaded from TMEM into registers while the MMAs of
//              the first half run;
//   layer 3    H2 = BF16(ReLU(D2 + b2)) stays in registers; the 4 outputs are
//              FP32 dot products with the BF16 rows of W3 (+ b3), summed per
//              warpgroup over its 64 columns and then across warpgroups in a
//              fixed order; the predictor y0 = y + e + (out_mean + out_std *
//              out) is written in FP64.
//
// The BF16 rounding points are those of the training kernels (inputs and
// weights of every layer).  Weights are packed once per call into the
// no-swizzle K-major canonical layout of the UMMA shared-memory descriptors
// (8-row x 16-byte core matrices; LBO = 128 B between core matrices along K,
// SBO = 16 B x K between 8-row groups) and copied to shared memory with bulk
// asynchronous copies.  Every wait is bounded: a wait that runs out sets an
// error flag that the host reads, the CTA stops issuing work, waits (bounded)
// for what it issued, frees its TMEM and returns.
#include <atomic>
#include <cuda_bf16.h>
#include <stdint.h>

#include "fsi_internal.cuh"
#include "tc_common.cuh"

namespace fsi {
namespace {

constexpr int NI = 112, NH = 256, NO = 4;
constexpr int64_t OFF_W1 = 0, OFF_b1 = OFF_W1 + NI * NH, OFF_W2 = OFF_b1 + NH,
                  OFF_b2 = OFF_W2 + NH * NH, OFF_W3 = OFF_b2 + NH, OFF_b3 = OFF_W3 + NH * NO;

constexpr int TM = 128;                         // nodes per tile (MMA M)
constexpr uint32_t KC1 = NI / 8, KC2 = 128 / 8;  // 16-byte K chunks: layer 1, half of layer 2
constexpr uint32_t SZ_W1 = NH * NI * 2;          // 57,344
constexpr uint32_t SZ_W2H = NH * 128 * 2;        // 65,536 (one K-half of W2)
constexpr uint32_t SZ_XH = TM * 128 * 2;         // 32,768 (X [128 x 112] or H1 half)
constexpr uint32_t OFF_SW1 = 0, OFF_SW2A = OFF_SW1 + SZ_W1, OFF_SW2B = OFF_SW2A + SZ_W2H,
                   OFF_SXH = OFF_SW2B + SZ_W2H, OFF_SW3 = OFF_SXH + SZ_XH,
                   OFF_SB1 = OFF_SW3 + NH * 16, OFF_SB2 = OFF_SB1 + NH * 4,
                   SMEM_BYTES = OFF_SB2 + NH * 4;  // 227,328
constexpr uint32_t PACKED_BYTES = SZ_W1 + 2 * SZ_W2H;  // 188,416
constexpr uint32_t TMEM_COLS = 512;
// Four warpgroups share every tile: warp w reads TMEM lanes 32 (w % 4) ..
// (the tile's node rows), so warpgroup g = w / 4 takes the same rows and its
// share of the columns: feature chunks [kChunk[g], kChunk[g + 1]), H1
// columns 32 g .. of each K-half, D2 columns 64 g .. of layer 3.
constexpr int kGroups = 4;
constexpr int kThreads = 128 * kGroups;
__constant__ int kChunk[kGroups + 1] = {0, 4, 8, 11, 14};

using namespace tc;

constexpr uint32_t kIdesc = idesc_bf16(TM, NH);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    tc::mma_bf16(d_tmem, a, b, kIdesc, acc);
}

// W1 [NI][NH] and W2 [NH][NH] (input-major, as trained) -> B operands
// [N = out][K = in] BF16 in the canonical layout: W1 (K = 112), then the two
// K-halves of W2 (K = 0..127, 128..255)
__global__ void pack_weights_kernel(const float *P, uint8_t *packed)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)NH * (NI + NH);
         e += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(e % NH);
        const int k = (int)(e / NH);
        __nv_bfloat16 v;
        uint32_t off;
        if (k < NI) {
            v = __float2bfloat16_rn(P[OFF_W1 + (int64_t)k * NH + n]);
            off = OFF_SW1 + kmaj(n, k, KC1);
        } else {
            const int k2 = k - NI;
            v = __float2bfloat16_rn(P[OFF_W2 + (int64_t)k2 * NH + n]);
            off = (k2 < 128 ? OFF_SW2A : OFF_SW2B) + kmaj(n, k2 & 127, KC2);
        }
        *reinterpret_cast<__nv_bfloat16 *>(packed + off) = v;
    }
}

struct TcArgs {
    int Nx, Ny, Nz;
    int64_t n;
    const float *P;  // FP32 parameters (biases, W3)
    const uint8_t *packed;
    const float *in_mean, *in_std, *out_mean, *out_std;
    const double *Vn, *y, *d1, *d2;
    double *y0;
    int *err;
};

__global__ void __launch_bounds__(kThreads, 1) mlp_predict_tc_kernel(const TcArgs a)
{
    extern __shared__ __align__(128) uint8_t sm[];
    __shared__ __align__(8) uint64_t bars[2];  // [0] weights, [1] MMA completion
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    __shared__ float smean[NI], sistd[NI];
    const int tid = threadIdx.x, warp = tid >> 5, row = tid & (TM - 1), grp = tid >> 7;
    const uint32_t s0 = smem_u32(sm);
    const uint32_t bar_w = smem_u32(&bars[0]), bar_m = smem_u32(&bars[1]);

    if (tid == 0) {
        abort_flag = 0;
        mbar_init(bar_w, 1);
        mbar_init(bar_m, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // small operands: W3 (BF16-rounded, one float4 per hidden unit), b1, b2
    float4 *sW3 = reinterpret_cast<float4 *>(sm + OFF_SW3);
    float *sb1 = reinterpret_cast<float *>(sm + OFF_SB1), *sb2 = reinterpret_cast<float *>(sm + OFF_SB2);
    for (int f = tid; f < NI; f += blockDim.x) {
        smean[f] = a.in_mean[f];
        sistd[f] = 1.0f / a.in_std[f];
    }
    for (int c = tid; c < NH; c += blockDim.x) {
        const float *w = a.P + OFF_W3 + (int64_t)c * NO;
        sW3[c] = make_float4(bf16r(w[0]), bf16r(w[1]), bf16r(w[2]), bf16r(w[3]));
        sb1[c] = a.P[OFF_b1 + c];
        sb2[c] = a.P[OFF_b2 + c];
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_holder;
    // weights: bulk asynchronous copies into shared memory, once per CTA
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_w),
                     "r"(PACKED_BYTES)
                     : "memory");
        for (uint32_t off = 0; off < PACKED_BYTES; off += 16384) {
            const uint32_t bytes = PACKED_BYTES - off < 16384 ? PACKED_BYTES - off : 16384;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    s0 + off),
                "l"(a.packed + off), "r"(bytes), "r"(bar_w)
                : "memory");
        }
    }
    uint32_t mma_phase = 0;
    bool mma_pending = false;  // a commit was issued and not yet observed
    const bool weights_ok = mbar_wait(bar_w, 0);
    bool ok = weights_ok;
    if (!ok) atomicExch(&abort_flag, 1);
    __syncthreads();
    const float b3[4] = {a.P[OFF_b3], a.P[OFF_b3 + 1], a.P[OFF_b3 + 2], a.P[OFF_b3 + 3]};
    const float om[4] = {a.out_mean[0], a.out_mean[1], a.out_mean[2], a.out_mean[3]};
    const float os[4] = {a.out_std[0], a.out_std[1], a.out_std[2], a.out_std[3]};
    const int nx = a.Nx + 1, ny = a.Ny + 1, nz = a.Nz + 1;
    const int64_t ntiles = (a.n + TM - 1) / TM;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    uint8_t *xh = sm + OFF_SXH;

    for (int64_t tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
        const int64_t node = tile * TM + row;
        const bool live = node < a.n;
        // ---- features -> X (BF16, canonical K-major, 14 chunks of 8 = two
        // stencil points each, the last one point and the extrapolant).  Group
        // g builds chunks [kChunk[g], kChunk[g + 1]).  The normalisation runs
        // in FP32 ((value - mean) * (1 / std)): the result is rounded to BF16
        // right away, and GB300's FP64 unit is ~70x slower.
        {
            int i = 0, j = 0, k = 0;
            if (live) {
                i = (int)(node % nx);
                j = (int)((node / nx) % ny);
                k = (int)(node / ((int64_t)nx * ny));
            }
            for (int c = kChunk[grp]; c < kChunk[grp + 1]; ++c) {
                float f8[8];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int s = 2 * c + h;
                    double raw[4] = {0.0, 0.0, 0.0, 0.0};
                    if (s < 27) {
                        const int ii = i + s % 3 - 1, jj = j + (s / 3) % 3 - 1, kk = k + s / 9 - 1;
                        const bool in = live && ii >= 0 && ii < nx && jj >= 0 && jj < ny &&
                                        kk >= 0 && kk < nz;
                        if (in) {
                            const int64_t nb = ii + (int64_t)nx * (jj + (int64_t)ny * kk);
                            const double2 v01 =
                                __ldg(reinterpret_cast<const double2 *>(a.Vn + 4 * nb));
                            raw[0] = v01.x;
                            raw[1] = v01.y;
                            raw[2] = __ldg(a.Vn + 4 * nb + 2);
                            raw[3] = __ldg(a.y + 4 * nb + 3);
                        }
                    } else if (live) {  // features 108..111: the extrapolant 2 d1 - d2
#pragma unroll
                        for (int q = 0; q < 4; ++q) raw[q] = 2.0 * a.d1[4 * node + q] - a.d2[4 * node + q];
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int f = 4 * s + q;
                        f8[4 * h + q] = live ? ((float)raw[q] - smean[f]) * sistd[f] : 0.0f;
                    }
                }
                const uint4 v = make_uint4(pack_bf16(f8[0], f8[1]), pack_bf16(f8[2], f8[3]),
                                           pack_bf16(f8[4], f8[5]), pack_bf16(f8[6], f8[7]));
                *reinterpret_cast<uint4 *>(xh + kmaj(row, 8 * c, KC1)) = v;
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        // ---- layer 1: D1 = X W1^T
        if (tid == 0) {
            fence_after();
            for (uint32_t ks = 0; ks < NI / 16; ++ks)
                mma_bf16(tmem + 0, sdesc(s0 + OFF_SXH + ks * 256, 128, KC1 * 128),
                         sdesc(s0 + OFF_SW1 + ks * 256, 128, KC1 * 128), ks > 0);
            mma_commit(bar_m);
        }
        mma_pending = true;
        ok = mbar_wait(bar_m, mma_phase);
        if (ok) {
            mma_phase ^= 1;
            mma_pending = false;
        } else {
            atomicExch(&abort_flag, 1);
        }
        __syncthreads();
        if (abort_flag) break;
        fence_after();
        // ---- H1, first K-half (columns 0..127) -> shared memory (aliases X):
        // group g converts columns 32 g .. 32 g + 31
        {
            float v[32];
            tmem_ld32(tmem + lane_base + 32 * grp, v);
#pragma unroll
            for (int q8 = 0; q8 < 4; ++q8) {
                float h[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int col = 32 * grp + 8 * q8 + t;
                    h[t] = fmaxf(v[8 * q8 + t] + sb1[col], 0.0f);
                }
                *reinterpret_cast<uint4 *>(xh + kmaj(row, 32 * grp + 8 * q8, KC2)) =
                    make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]),
                               pack_bf16(h[6], h[7]));
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            for (uint32_t ks = 0; ks < 8; ++ks)
                mma_bf16(tmem + NH, sdesc(s0 + OFF_SXH + ks * 256, 128, KC2 * 128),
                         sdesc(s0 + OFF_SW2A + ks * 256, 128, KC2 * 128), ks > 0);
            mma_commit(bar_m);
        }
        // second K-half of H1 (group g: columns 128 + 32 g ..) into registers
        // while those MMAs run
        uint32_t hp[16];
        {
            float v[32];
            tmem_ld32(tmem + lane_base + 128 + 32 * grp, v);
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int col = 128 + 32 * grp + 2 * t;
                hp[t] = pack_bf16(fmaxf(v[2 * t] + sb1[col], 0.0f),
                                  fmaxf(v[2 * t + 1] + sb1[col + 1], 0.0f));
            }
        }
        mma_pending = true;
        ok = mbar_wait(bar_m, mma_phase);
        if (ok) {
            mma_phase ^= 1;
            mma_pending = false;
        } else {
            atomicExch(&abort_flag, 1);
        }
        __syncthreads();
        if (abort_flag) break;
#pragma unroll
        for (int q8 = 0; q8 < 4; ++q8)
            *reinterpret_cast<uint4 *>(xh + kmaj(row, 32 * grp + 8 * q8, KC2)) =
                make_uint4(hp[4 * q8], hp[4 * q8 + 1], hp[4 * q8 + 2], hp[4 * q8 + 3]);
        fence_async_smem();
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            for (uint32_t ks = 0; ks < 8; ++ks)
                mma_bf16(tmem + NH, sdesc(s0 + OFF_SXH + ks * 256, 128, KC2 * 128),
                         sdesc(s0 + OFF_SW2B + ks * 256, 128, KC2 * 128), 1);
            mma_commit(bar_m);
        }
        mma_pending = true;
        ok = mbar_wait(bar_m, mma_phase);
        if (ok) {
            mma_phase ^= 1;
            mma_pending = false;
        } else {
            atomicExch(&abort_flag, 1);
        }
        __syncthreads();
        if (abort_flag) break;
        fence_after();
        // ---- layer 3: group g sums D2 columns 64 g .. 64 g + 63; groups 1..3
        // leave their partial sums in the X buffer (free now), group 0 adds
        // them in group order and writes the predictor
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            float v[32];
            tmem_ld32(tmem + lane_base + NH + 64 * grp + 32 * c, v);
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                const int col = 64 * grp + 32 * c + t;
                const float h = bf16r(fmaxf(v[t] + sb2[col], 0.0f));
                const float4 w = sW3[col];
                o[0] = fmaf(h, w.x, o[0]);
                o[1] = fmaf(h, w.y, o[1]);
                o[2] = fmaf(h, w.z, o[2]);
                o[3] = fmaf(h, w.w, o[3]);
            }
        }
        float4 *part = reinterpret_cast<float4 *>(xh);
        if (grp > 0) part[(grp - 1) * TM + row] = make_float4(o[0], o[1], o[2], o[3]);
        __syncthreads();
        if (grp == 0) {
#pragma unroll
            for (int g = 1; g < kGroups; ++g) {
                const float4 p = part[(g - 1) * TM + row];
                o[0] += p.x;
                o[1] += p.y;
                o[2] += p.z;
                o[3] += p.w;
            }
            if (live)
                for (int c = 0; c < 4; ++c) {
                    const int64_t qn = 4 * node + c;
                    const double e = 2.0 * a.d1[qn] - a.d2[qn];
                    const float out = o[c] + b3[c];
                    a.y0[qn] = a.y[qn] + e + ((double)om[c] + (double)os[c] * (double)out);
                }
        }
        // the next tile overwrites X (read by the finished MMAs and by group 0
        // above) and D1
        fence_before();
        __syncthreads();
    }
    if (abort_flag && tid == 0) atomicExch(a.err, 1);
    // nothing may still be in flight when the TMEM is freed: a CTA that gave
    // up waits (bounded) for its last commit before releasing
    if (abort_flag) {
        if (mma_pending) mbar_wait(bar_m, mma_phase);
        if (!weights_ok) mbar_wait(bar_w, 0);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// Self-test of the bounded wait: one thread waits, with the production wait
// loop, on an mbarrier that expects one arrival that never comes.  The wait
// must run out; the kernel then raises the error flag and returns.
__global__ void wait_selftest_kernel(int *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
        mbar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait(b, 0)) atomicExch(err, 1);
    }
}

}  // namespace

size_t mlp_tc_packed_bytes() { return PACKED_BYTES; }

fsi_status mlp_predict_tc(cudaStream_t s, int device, const fsi_grid &g, int64_t n,
                          const float *params, const float *in_mean, const float *in_std,
                          const float *out_mean, const float *out_std, const double *Vn,
                          const double *y, const double *d1, const double *d2, double *y0,
                          void *packed, int *dev_err)
{
    if (n <= 0) return FSI_OK;
    // the attribute is per device; setting it twice (two threads racing on
    // the first call) is harmless, the flags only skip later calls
    static std::atomic<bool> attr_set[64];
    if (device < 0 || device >= 64 || !attr_set[device].load(std::memory_order_acquire)) {
        FSI_CUDA(cudaFuncSetAttribute(mlp_predict_tc_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES),
                 "cudaFuncSetAttribute");
        if (device >= 0 && device < 64) attr_set[device].store(true, std::memory_order_release);
    }
    const int sms = sm_count();
    pack_weights_kernel<<<sm_count() * 4, 256, 0, s>>>(params, (uint8_t *)packed);
    FSI_TRY(check_launch("pack weights"));
    TcArgs a{g.N[0], g.N[1], g.N[2], n, params, (const uint8_t *)packed, in_mean, in_std,
             out_mean, out_std, Vn, y, d1, d2, y0, dev_err};
    const int64_t tiles = (n + TM - 1) / TM;
    const int grid = (int)(tiles < sms ? tiles : sms);
    mlp_predict_tc_kernel<<<grid, kThreads, SMEM_BYTES, s>>>(a);
    // asynchronous: a wait that ran out stays flagged in dev_err until the
    // handle's next check (fsi_mlp_check, fsi_mlp_guess)
    return check_launch("tensor-core predict");
}

}  // namespace fsi

extern "C" fsi_status fsi_wait_selftest(int device, int *timed_out, double *seconds)
{
    using namespace fsi;
    if (!timed_out || !seconds) return set_error(FSI_ERR_ARG, "fsi_wait_selftest: NULL output");
    FSI_DEVICE(device);
    int *err = nullptr;
    FSI_CUDA(cudaMalloc(&err, sizeof(int)), "cudaMalloc");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemset(err, 0, sizeof(int));
    cudaEventRecord(e0);
    wait_selftest_kernel<<<1, 32>>>(err);
    cudaEventRecord(e1);
    fsi_status st = check_launch("wait self-test");
    int h = 0;
    if (st == FSI_OK) st = check_cuda(cudaMemcpy(&h, err, sizeof h, cudaMemcpyDeviceToHost),
                                      "memcpy");
    float ms = 0.0f;
    if (st == FSI_OK) st = check_cuda(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(err);
    *timed_out = h;
    *seconds = ms * 1e-3;
    return st;
}
