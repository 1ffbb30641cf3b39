// batch.cu -- many independent instances of uneven size in one pass (an
// extension; the paper has no counterpart): the point location and cell
// table, the residual, the Jacobian apply, interpolation and spreading of
// every instance run as persistent grids that walk a prefix sum of
// (instance, work item) pairs, so small grids no longer leave SMs idle and the
// whole step is a handful of launches, which one CUDA graph replays.  A
// native autotuner picks the brick shape and the persistent grid size by
// timing candidates on the actual batch.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "dlm_device.cuh"
#include "vms_device.cuh"

namespace fsi {
namespace {

template <typename T> struct DlmDesc {
    dlmd::GridArgs g;
    int64_t m, E;
    const int32_t *elem, *start, *perm;
    const T *xi, *lam, *w;
    const vec4<T> *U;
    T *u, *F, *S;
    // batched location: raw points (null when the item brings its own
    // table), per-cell counters [E+1], scan tile sums [ntiles] (+ the count
    // of CTA-sorted cells) and (point, cell) pairs [m]; the step then writes
    // elem, xi, start and perm
    const double *X;
    int32_t *fill, *tiles;
    int2 *pairs;
    int64_t ntiles;
};

// cells of more points than this are sorted by a CTA instead of the rank
// pass (whose work per point grows with its cell's size)
constexpr int kBatchRankMax = 512;

constexpr int kChunk = 256;  // nodes / points per work item; 8 cell segments per item

__device__ __forceinline__ int find_instance(const int64_t *prefix, int count, int64_t item)
{
    int lo = 0, hi = count;  // prefix[lo] <= item < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename T, bool JAC>
__global__ void __launch_bounds__(256) batch_brick_kernel(const vmsd::VmsArgs<T> *desc,
                                                          const int64_t *prefix, int count)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    auto *rel = reinterpret_cast<vec4<T> *>(smem_raw);
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        vmsd::brick_body<T, JAC>(desc[inst], (int)(item - prefix[inst]), rel);
        __syncthreads();  // rel is reused by the next brick
    }
}

template <typename T>
__global__ void batch_gather_kernel(const vmsd::VmsArgs<T> *desc, const int64_t *prefix, int count)
{
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const vmsd::VmsArgs<T> &P = desc[inst];
        const int n = (P.Nx + 1) * (P.Ny + 1) * (P.Nz + 1);
        const int64_t node = (item - prefix[inst]) * kChunk + threadIdx.x;
        if (node < n) vmsd::gather_node(P, (int)node);
    }
}

// ---- batched location and cell table (the bodies of dlm_device.cuh over
// the instances' prefix sums; instances without raw points are skipped)
template <typename T>
__global__ void batch_clear_kernel(const DlmDesc<T> *desc, const int64_t *prefix, int count)
{
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const DlmDesc<T> &D = desc[inst];
        const int64_t c = (item - prefix[inst]) * kChunk + threadIdx.x;
        if (D.X && c <= D.E) D.fill[c] = 0;
        if (D.X && c == 0) D.tiles[D.ntiles] = 0;  // count of CTA-sorted cells
    }
}

template <typename T>
__global__ void batch_locate_kernel(const DlmDesc<T> *desc, const int64_t *prefix, int count)
{
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const DlmDesc<T> &D = desc[inst];
        const int64_t b = (item - prefix[inst]) * kChunk + threadIdx.x;
        if (D.X && b < D.m) {
            const int e = dlmd::locate_point<T>(D.g, b, D.X, const_cast<int32_t *>(D.elem),
                                                const_cast<T *>(D.xi));
            // the count the cell had before this point (outside points count
            // in the tail cell E): the point's slot in its cell's slice
            const_cast<int32_t *>(D.perm)[b] = atomicAdd(D.fill + (e >= 0 ? (int64_t)e : D.E), 1);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) batch_scan_tiles_kernel(const DlmDesc<T> *desc,
                                                                const int64_t *prefix, int count)
{
    __shared__ int warp_sums[32];
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const DlmDesc<T> &D = desc[inst];
        if (D.X)  // uniform over the block
            dlmd::scan_tile(D.E, D.fill, const_cast<int32_t *>(D.start), D.tiles,
                            item - prefix[inst], warp_sums);
        __syncthreads();  // warp_sums is reused by the next tile
    }
}

// one CTA per instance scans that instance's tile sums
template <typename T>
__global__ void __launch_bounds__(1024) batch_scan_totals_kernel(const DlmDesc<T> *desc, int count)
{
    __shared__ int warp_sums[32];
    __shared__ int carry;
    for (int inst = blockIdx.x; inst < count; inst += gridDim.x) {
        const DlmDesc<T> &D = desc[inst];
        if (D.X) dlmd::scan_totals_block(D.ntiles, D.tiles, warp_sums, &carry);
        __syncthreads();
    }
}

template <typename T>
__global__ void batch_scan_add_kernel(const DlmDesc<T> *desc, const int64_t *prefix, int count)
{
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const DlmDesc<T> &D = desc[inst];
        if (D.X)
            dlmd::scan_add_tile(D.E, const_cast<int32_t *>(D.start), D.tiles, item - prefix[inst]);
    }
}

// (point, cell) pairs at their arrival slots (the single-mesh table's
// scatter, per instance)
template <typename T>
__global__ void batch_scatter_kernel(const DlmDesc<T> *desc, const int64_t *prefix, int count)
{
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const DlmDesc<T> &D = desc[inst];
        const int64_t b = (item - prefix[inst]) * kChunk + threadIdx.x;
        if (D.X && b < D.m) {
            const int e = D.elem[b];
            const int c = e >= 0 ? e : (int)D.E;
            const int64_t pos = (int64_t)D.start[c] + D.perm[b];
            if (pos >= 0 && pos < D.m) D.pairs[pos] = make_int2((int)b, c);
        }
    }
}

// each slot's final place: the number of its cell's points with a smaller
// index (cells of more than kBatchRankMax points go to the dense list in the
// spent counters, counted in tiles[ntiles])
template <typename T>
__global__ void batch_rank_kernel(const DlmDesc<T> *desc, const int64_t *prefix, int count)
{
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const DlmDesc<T> &D = desc[inst];
        const int64_t k = (item - prefix[inst]) * kChunk + threadIdx.x;
        if (!D.X || k >= D.m) continue;
        const int2 p = D.pairs[k];
        const int lo = D.start[p.y];
        const int hi = p.y < D.E ? D.start[p.y + 1] : (int)D.m;
        if (hi - lo > kBatchRankMax) {
            if (k == lo) D.fill[atomicAdd(D.tiles + D.ntiles, 1)] = p.y;
            continue;
        }
        int r = 0;
        for (int j = lo; j < hi; ++j) r += D.pairs[j].x < p.x;
        const_cast<int32_t *>(D.perm)[lo + r] = p.x;
    }
}

// the listed cells, one CTA per cell: the pairs' points into perm, then a
// bitonic sort in shared memory (or one lane's shell sort beyond
// kBlockSortMax points)
template <typename T>
__global__ void __launch_bounds__(1024) batch_dense_sort_kernel(const DlmDesc<T> *desc, int count)
{
    extern __shared__ int32_t sort_sh[];
    // the instances' lists read as one: CTA b takes entries b, b + grid, ...
    int64_t g = blockIdx.x, base = 0;
    for (int inst = 0; inst < count; ++inst) {
        const DlmDesc<T> &D = desc[inst];
        if (!D.X) continue;
        const int n = D.tiles[D.ntiles];
        for (; g < base + n; g += gridDim.x) {
            const int c = D.fill[g - base];
            const int lo = D.start[c];
            const int len = (c < D.E ? D.start[c + 1] : (int)D.m) - lo;
            int32_t *perm = const_cast<int32_t *>(D.perm);
            for (int i = threadIdx.x; i < len; i += blockDim.x) perm[lo + i] = D.pairs[lo + i].x;
            __syncthreads();
            dlmd::block_sort_cell(D.E, D.m, D.start, perm, c, sort_sh);
        }
        base += n;
    }
}

template <typename T>
__global__ void cast_xi_kernel(int64_t n, const double *src, T *dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

template <typename T>
__global__ void batch_interp_kernel(const DlmDesc<T> *desc, const int64_t *prefix, int count)
{
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const DlmDesc<T> &D = desc[inst];
        if constexpr (std::is_same<T, float>::value) {
            // the chunk's kChunk points in two halves, two lanes per point
            // (the single-mesh FP32 kernel's arithmetic)
            for (int half = 0; half < 2; ++half) {
                const int64_t b = (item - prefix[inst]) * kChunk + half * (kChunk / 2) +
                                  (threadIdx.x >> 1);
                dlmd::interp_point_pair<T>(D.g, b, b < D.m, D.elem, D.xi, D.U, D.u);
            }
        } else {
            const int64_t b = (item - prefix[inst]) * kChunk + threadIdx.x;
            if (b < D.m) dlmd::interp_point<T>(D.g, b, D.elem, D.xi, D.U, D.u);
        }
    }
}

template <typename T>
__global__ void batch_spread_cells_kernel(const DlmDesc<T> *desc, const int64_t *prefix,
                                          int count)
{
    const int64_t total = prefix[count];
    const int warp = threadIdx.x >> 5;
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const DlmDesc<T> &D = desc[inst];
        const int64_t c0 = ((item - prefix[inst]) * 8 + warp) * dlmd::kSpreadSeg;
        if (c0 < D.E) dlmd::spread_cells_segment<T>(D.E, c0, D.xi, D.start, D.perm, D.lam, D.w, D.S);
    }
}

template <typename T>
__global__ void batch_spread_nodes_kernel(const DlmDesc<T> *desc, const int64_t *prefix,
                                          int count)
{
    const int64_t total = prefix[count];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        const int inst = find_instance(prefix, count, item);
        const DlmDesc<T> &D = desc[inst];
        const int NX1 = D.g.Nx + 1, NY1 = D.g.Ny + 1;
        const int n = NX1 * NY1 * (D.g.Nz + 1);
        const int64_t node = (item - prefix[inst]) * kChunk + threadIdx.x;
        if (node < n) {
            const int nd = (int)node;
            dlmd::spread_node<T>(D.g, nd % NX1, (nd / NX1) % NY1, nd / (NX1 * NY1), D.start, D.S,
                                 D.F, 0);
        }
    }
}

}  // namespace
}  // namespace fsi

struct fsi_batch {
    int device;
    cudaStream_t stream;
    fsi_prec prec;
    int count;
    std::vector<fsi_mesh *> meshes;
    std::vector<fsi_batch_item> items;
    fsi::Brick brick;
    int ctas_per_sm;
    int sms;
    // device data
    void *desc_res, *desc_jac, *desc_dlm;                      // descriptors
    // [kRows][count+1]: bricks, node chunks, point chunks, spreading cell items,
    // counter chunks (E+1 cells), scan tiles
    int64_t *prefix;
    void *blocks;
    size_t blocks_bytes;
    void *spread;
    size_t spread_bytes;
    // batched location: per-cell counters and scan tile sums of every
    // instance that brings raw points; FP64 xi of one instance for the
    // per-instance path of an FP32 batch
    void *loc;
    size_t loc_bytes;
    double *xi64;
    size_t xi64_bytes;
    bool locate;
    int64_t totals[6];
    // CUDA graph of one batched step
    cudaGraph_t graph;
    cudaGraphExec_t graph_exec;
};

namespace fsi {
namespace {

constexpr int kRows = 6;

// (Re)build descriptors and scratch for the batch's current brick shape.
template <typename T> fsi_status build_batch(fsi_batch *b)
{
    const int C = b->count;
    std::vector<vmsd::VmsArgs<T>> res(C), jac(C);
    std::vector<DlmDesc<T>> dlm(C);
    std::vector<int64_t> pre(kRows * (C + 1), 0);
    size_t blocks_need = 0, spread_need = 0, loc_need = 0, xi64_need = 0;
    std::vector<size_t> boff(C), soff(C), loff(C);
    for (int i = 0; i < C; ++i) {
        fsi_mesh *m = b->meshes[i];
        boff[i] = blocks_need;
        blocks_need += vms_scratch_bytes_for(m, b->brick, sizeof(T));
        blocks_need = (blocks_need + 255) / 256 * 256;
        soff[i] = spread_need;
        spread_need += (size_t)m->n_elems * 24 * sizeof(T);
        spread_need = (spread_need + 255) / 256 * 256;
        loff[i] = loc_need;
        if (b->items[i].X) {
            loc_need += (size_t)(m->n_elems + 1 + dlmd::cell_tiles(m->n_elems) + 1) * sizeof(int32_t);
            loc_need = (loc_need + 255) / 256 * 256;
            loc_need += (size_t)b->items[i].m * sizeof(int2);  // the pairs
            loc_need = (loc_need + 255) / 256 * 256;
            xi64_need = std::max(xi64_need, (size_t)b->items[i].m * 3 * sizeof(double));
        }
    }
    if (loc_need > b->loc_bytes) {
        cudaFree(b->loc);
        b->loc = nullptr;
        b->loc_bytes = 0;
        FSI_CUDA(cudaMalloc(&b->loc, loc_need), "batch location scratch");
        b->loc_bytes = loc_need;
    }
    if (sizeof(T) != sizeof(double) && xi64_need > b->xi64_bytes) {
        cudaFree(b->xi64);
        b->xi64 = nullptr;
        b->xi64_bytes = 0;
        FSI_CUDA(cudaMalloc(&b->xi64, xi64_need), "batch xi scratch");
        b->xi64_bytes = xi64_need;
    }
    if (blocks_need > b->blocks_bytes) {
        cudaFree(b->blocks);
        b->blocks = nullptr;
        b->blocks_bytes = 0;
        FSI_CUDA(cudaMalloc(&b->blocks, blocks_need), "batch block scratch");
        b->blocks_bytes = blocks_need;
    }
    if (spread_need > b->spread_bytes) {
        cudaFree(b->spread);
        b->spread = nullptr;
        b->spread_bytes = 0;
        FSI_CUDA(cudaMalloc(&b->spread, spread_need), "batch spread scratch");
        b->spread_bytes = spread_need;
    }
    for (int i = 0; i < C; ++i) {
        fsi_mesh *m = b->meshes[i];
        const fsi_batch_item &it = b->items[i];
        res[i] = vmsd::make_args<T>(m, b->brick, it.U, it.A, it.f, nullptr, it.R);
        jac[i] = vmsd::make_args<T>(m, b->brick, it.U, it.A, it.f, it.x, it.Jx);
        res[i].blocks = jac[i].blocks = (vec4<T> *)((char *)b->blocks + boff[i]);
        DlmDesc<T> &D = dlm[i];
        D.g.Nx = m->grid.N[0];
        D.g.Ny = m->grid.N[1];
        D.g.Nz = m->grid.N[2];
        D.g.x0 = m->grid.x0[0];
        D.g.y0 = m->grid.x0[1];
        D.g.z0 = m->grid.x0[2];
        D.g.hx = m->grid.h[0];
        D.g.hy = m->grid.h[1];
        D.g.hz = m->grid.h[2];
        dlmd::set_reciprocals(D.g);
        D.m = it.m;
        D.E = m->n_elems;
        D.elem = it.elem;
        D.start = it.cell_start;
        D.perm = it.perm;
        D.xi = (const T *)it.xi;
        D.lam = (const T *)it.lam;
        D.w = (const T *)it.w;
        D.U = (const vec4<T> *)it.U;
        D.u = (T *)it.u;
        D.F = (T *)it.F;
        D.S = (T *)((char *)b->spread + soff[i]);
        D.X = it.X;
        D.ntiles = dlmd::cell_tiles(m->n_elems);
        D.fill = it.X ? (int32_t *)((char *)b->loc + loff[i]) : nullptr;
        D.tiles = it.X ? D.fill + m->n_elems + 1 : nullptr;
        if (it.X) {
            const size_t off = ((size_t)(m->n_elems + 1 + D.ntiles + 1) * sizeof(int32_t) + 255) /
                               256 * 256;
            D.pairs = (int2 *)((char *)b->loc + loff[i] + off);
        } else {
            D.pairs = nullptr;
        }
        const int64_t nb = (int64_t)res[i].nbx * res[i].nby * res[i].nbz;
        pre[0 * (C + 1) + i + 1] = pre[0 * (C + 1) + i] + nb;
        pre[1 * (C + 1) + i + 1] = pre[1 * (C + 1) + i] + (m->n_nodes + kChunk - 1) / kChunk;
        pre[2 * (C + 1) + i + 1] = pre[2 * (C + 1) + i] + (it.m + kChunk - 1) / kChunk;
        pre[3 * (C + 1) + i + 1] =
            pre[3 * (C + 1) + i] +
            ((m->n_elems + dlmd::kSpreadSeg - 1) / dlmd::kSpreadSeg + 7) / 8;  // 8 segments per item
        const int64_t cells = it.X ? (m->n_elems + 1 + kChunk - 1) / kChunk : 0;
        pre[4 * (C + 1) + i + 1] = pre[4 * (C + 1) + i] + cells;
        pre[5 * (C + 1) + i + 1] = pre[5 * (C + 1) + i] + (it.X ? D.ntiles : 0);
    }
    for (int k = 0; k < kRows; ++k) b->totals[k] = pre[k * (C + 1) + C];
    cudaStream_t s = b->stream;
    FSI_CUDA(cudaMemcpyAsync(b->desc_res, res.data(), C * sizeof(res[0]), cudaMemcpyHostToDevice, s),
             "descriptor upload");
    FSI_CUDA(cudaMemcpyAsync(b->desc_jac, jac.data(), C * sizeof(jac[0]), cudaMemcpyHostToDevice, s),
             "descriptor upload");
    FSI_CUDA(cudaMemcpyAsync(b->desc_dlm, dlm.data(), C * sizeof(dlm[0]), cudaMemcpyHostToDevice, s),
             "descriptor upload");
    FSI_CUDA(cudaMemcpyAsync(b->prefix, pre.data(), pre.size() * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s),
             "prefix upload");
    FSI_CUDA(cudaStreamSynchronize(s), "sync");
    if (b->graph_exec) {
        cudaGraphExecDestroy(b->graph_exec);
        b->graph_exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    return FSI_OK;
}

// phases of a batched step: 1 residual, 2 Jacobian apply, 4 interpolation and
// spreading, 8 location and cell table (instances with raw points)
constexpr int kAllPhases = 15;

int persistent_grid(const fsi_batch *b, int64_t items)
{
    int64_t g = (int64_t)b->sms * b->ctas_per_sm;
    if (items < g) g = items;
    return (int)(g < 1 ? 1 : g);
}

// The batched step: residual, Jacobian apply, interpolation, spreading.
template <typename T> fsi_status run_batched(fsi_batch *b, int phases)
{
    cudaStream_t s = b->stream;
    const int C = b->count;
    const int64_t *pre = b->prefix;
    const size_t smem = (size_t)vmsd::rel_records(b->brick.bx * b->brick.by * b->brick.bz) *
                        sizeof(vec4<T>);
    if ((phases & 8) && b->locate) {
        const DlmDesc<T> *dd = (const DlmDesc<T> *)b->desc_dlm;
        batch_clear_kernel<T><<<persistent_grid(b, b->totals[4]), kChunk, 0, s>>>(
            dd, pre + 4 * (C + 1), C);
        if (b->totals[2] > 0)
            batch_locate_kernel<T><<<persistent_grid(b, b->totals[2]), kChunk, 0, s>>>(
                dd, pre + 2 * (C + 1), C);
        batch_scan_tiles_kernel<T><<<persistent_grid(b, b->totals[5]), 1024, 0, s>>>(
            dd, pre + 5 * (C + 1), C);
        batch_scan_totals_kernel<T><<<std::min(C, b->sms * 2), 1024, 0, s>>>(dd, C);
        batch_scan_add_kernel<T><<<persistent_grid(b, b->totals[5]), 256, 0, s>>>(
            dd, pre + 5 * (C + 1), C);
        if (b->totals[2] > 0) {
            batch_scatter_kernel<T><<<persistent_grid(b, b->totals[2]), kChunk, 0, s>>>(
                dd, pre + 2 * (C + 1), C);
            batch_rank_kernel<T><<<persistent_grid(b, b->totals[2]), kChunk, 0, s>>>(
                dd, pre + 2 * (C + 1), C);
            const int smem = dlmd::kBlockSortMax * (int)sizeof(int32_t);
            FSI_TRY(set_smem_limit((const void *)batch_dense_sort_kernel<T>, smem));
            batch_dense_sort_kernel<T><<<b->sms, 1024, smem, s>>>(dd, C);
        }
        FSI_TRY(check_launch("batched location kernels"));
    }
    if (phases & 1) {
        batch_brick_kernel<T, false><<<persistent_grid(b, b->totals[0]), b->brick.threads, smem, s>>>(
            (const vmsd::VmsArgs<T> *)b->desc_res, pre, C);
        batch_gather_kernel<T><<<persistent_grid(b, b->totals[1]), kChunk, 0, s>>>(
            (const vmsd::VmsArgs<T> *)b->desc_res, pre + (C + 1), C);
    }
    if (phases & 2) {
        batch_brick_kernel<T, true><<<persistent_grid(b, b->totals[0]), b->brick.threads, smem, s>>>(
            (const vmsd::VmsArgs<T> *)b->desc_jac, pre, C);
        batch_gather_kernel<T><<<persistent_grid(b, b->totals[1]), kChunk, 0, s>>>(
            (const vmsd::VmsArgs<T> *)b->desc_jac, pre + (C + 1), C);
    }
    if (phases & 4) {
        if (b->totals[2] > 0)
            batch_interp_kernel<T><<<persistent_grid(b, b->totals[2]), kChunk, 0, s>>>(
                (const DlmDesc<T> *)b->desc_dlm, pre + 2 * (C + 1), C);
        batch_spread_cells_kernel<T><<<persistent_grid(b, b->totals[3]), 256, 0, s>>>(
            (const DlmDesc<T> *)b->desc_dlm, pre + 3 * (C + 1), C);
        batch_spread_nodes_kernel<T><<<persistent_grid(b, b->totals[1]), kChunk, 0, s>>>(
            (const DlmDesc<T> *)b->desc_dlm, pre + (C + 1), C);
    }
    return check_launch("batched kernels");
}

fsi_status run_per_instance(fsi_batch *b, int phases)
{
    for (int i = 0; i < b->count; ++i) {
        fsi_mesh *m = b->meshes[i];
        const fsi_batch_item &it = b->items[i];
        cudaStream_t saved = m->stream;
        m->stream = b->stream;
        fsi::Brick bsaved[2] = {m->brick[0][b->prec], m->brick[1][b->prec]};
        m->brick[0][b->prec] = m->brick[1][b->prec] = b->brick;
        fsi_status st = FSI_OK;
        if ((phases & 8) && it.X) {
            // FP64 xi straight into the item, or through the batch's FP64
            // scratch and a rounding copy for an FP32 batch
            double *xi = b->prec == FSI_F64 ? (double *)it.xi : b->xi64;
            st = fsi_locate(m, it.m, it.X, const_cast<int32_t *>(it.elem), xi,
                            const_cast<int32_t *>(it.cell_start), const_cast<int32_t *>(it.perm),
                            nullptr, 0);
            if (st == FSI_OK && b->prec != FSI_F64 && it.m > 0) {
                cast_xi_kernel<float><<<sm_count() * 4, 256, 0, m->stream>>>(
                    3 * it.m, b->xi64, (float *)const_cast<void *>(it.xi));
                st = check_launch("xi rounding kernel");
            }
        }
        if (st == FSI_OK && (phases & 1)) st = fsi_residual(m, b->prec, it.U, it.A, it.f, it.R);
        if (st == FSI_OK && (phases & 2))
            st = fsi_jacobian_apply(m, b->prec, it.U, it.A, it.f, it.x, it.Jx);
        if (st == FSI_OK && (phases & 4)) {
            st = fsi_dlm_interp(m, b->prec, it.m, it.elem, it.xi, it.U, it.u);
            if (st == FSI_OK)
                st = fsi_dlm_spread(m, b->prec, it.m, it.elem, it.xi, it.cell_start, it.perm,
                                    it.lam, it.w, it.F, 0);
        }
        m->brick[0][b->prec] = bsaved[0];
        m->brick[1][b->prec] = bsaved[1];
        m->stream = saved;
        FSI_TRY(st);
    }
    return FSI_OK;
}

fsi_status set_smem_attr(fsi_prec prec)
{
    const int bytes = 200 * 1024;
    if (prec == FSI_F64) {
        FSI_TRY(set_smem_limit((const void *)batch_brick_kernel<double, false>, bytes));
        FSI_TRY(set_smem_limit((const void *)batch_brick_kernel<double, true>, bytes));
    } else {
        FSI_TRY(set_smem_limit((const void *)batch_brick_kernel<float, false>, bytes));
        FSI_TRY(set_smem_limit((const void *)batch_brick_kernel<float, true>, bytes));
    }
    return FSI_OK;
}

fsi_status run_mode(fsi_batch *b, int mode, int phases)
{
    if (mode == FSI_BATCH_PER_INSTANCE) return run_per_instance(b, phases);
    FSI_TRY(set_smem_attr(b->prec));
    if (mode == FSI_BATCH_PERSISTENT)
        return b->prec == FSI_F64 ? run_batched<double>(b, phases) : run_batched<float>(b, phases);
    // CUDA graph of the whole batched step (all phases), captured on first use
    if (!b->graph_exec) {
        if (b->stream == nullptr)
            return set_error(FSI_ERR_ARG, "graph mode needs a non-default stream");
        FSI_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal),
                 "begin capture");
        fsi_status st = b->prec == FSI_F64 ? run_batched<double>(b, kAllPhases)
                                           : run_batched<float>(b, kAllPhases);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        FSI_TRY(st);
        FSI_CUDA(e, "end capture");
        b->graph = g;
        FSI_CUDA(cudaGraphInstantiate(&b->graph_exec, g, 0), "graph instantiate");
    }
    return check_cuda(cudaGraphLaunch(b->graph_exec, b->stream), "graph launch");
}

// seconds per run of `mode` (events, best of reps)
fsi_status time_mode(fsi_batch *b, int mode, int phases, int reps, double *out)
{
    cudaEvent_t e0, e1;
    FSI_CUDA(cudaEventCreate(&e0), "event");
    FSI_CUDA(cudaEventCreate(&e1), "event");
    double best = 1e30;
    fsi_status st = run_mode(b, mode, phases);  // warm-up
    for (int r = 0; st == FSI_OK && r < reps; ++r) {
        cudaEventRecord(e0, b->stream);
        st = run_mode(b, mode, phases);
        cudaEventRecord(e1, b->stream);
        if (st == FSI_OK) st = check_cuda(cudaEventSynchronize(e1), "event sync");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms * 1e-3 < best) best = ms * 1e-3;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = best;
    return st;
}

const fsi::Brick kBrickCandidates[] = {
    {8, 8, 4, 256}, {8, 4, 4, 128}, {4, 4, 4, 64}, {16, 4, 4, 256}, {8, 8, 2, 128},
    {16, 8, 2, 256}, {4, 4, 8, 128}, {8, 4, 8, 256},
};

}  // namespace
}  // namespace fsi

using namespace fsi;

extern "C" {

fsi_status fsi_batch_create(fsi_mesh *const *meshes, const fsi_batch_item *items, int count,
                            fsi_prec prec, void *cuda_stream, fsi_batch **out)
{
    if (!out) return set_error(FSI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!meshes || !items || count < 1) return set_error(FSI_ERR_ARG, "empty batch");
    if (prec != FSI_F64 && prec != FSI_F32) return set_error(FSI_ERR_ARG, "bad precision");
    const int device = meshes[0] ? meshes[0]->device : -1;
    for (int i = 0; i < count; ++i) {
        if (!meshes[i]) return set_error(FSI_ERR_ARG, "mesh %d is NULL", i);
        if (meshes[i]->coords64 || meshes[i]->tet)
            return set_error(FSI_ERR_ARG, "mesh %d: the batch runs uniform grids only", i);
        if (meshes[i]->device != device)
            return set_error(FSI_ERR_ARG, "all meshes of a batch must be on one device");
        const fsi_batch_item &it = items[i];
        if (!it.U || !it.A || !it.x || !it.R || !it.Jx || !it.F || !it.cell_start)
            return set_error(FSI_ERR_ARG, "batch item %d: NULL array", i);
        if (it.m < 0 || it.m >= INT32_MAX ||
            (it.m > 0 && (!it.elem || !it.xi || !it.perm || !it.lam || !it.u)))
            return set_error(FSI_ERR_ARG, "batch item %d: bad point arrays", i);
    }
    FSI_DEVICE(device);
    fsi_batch *b = new (std::nothrow) fsi_batch();
    if (!b) return set_error(FSI_ERR_OOM, "host allocation failed");
    b->device = device;
    b->stream = (cudaStream_t)cuda_stream;
    b->prec = prec;
    b->count = count;
    b->meshes.assign(meshes, meshes + count);
    b->items.assign(items, items + count);
    for (int i = 0; i < count; ++i) b->locate = b->locate || items[i].X != nullptr;
    b->brick = Brick{8, 8, 4, 256};
    b->ctas_per_sm = 2;
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device);
    const size_t vsz = prec == FSI_F64 ? sizeof(vmsd::VmsArgs<double>) : sizeof(vmsd::VmsArgs<float>);
    const size_t dsz = prec == FSI_F64 ? sizeof(DlmDesc<double>) : sizeof(DlmDesc<float>);
    fsi_status st = check_cuda(cudaMalloc(&b->desc_res, count * vsz), "descriptors");
    if (st == FSI_OK) st = check_cuda(cudaMalloc(&b->desc_jac, count * vsz), "descriptors");
    if (st == FSI_OK) st = check_cuda(cudaMalloc(&b->desc_dlm, count * dsz), "descriptors");
    if (st == FSI_OK)
        st = check_cuda(cudaMalloc(&b->prefix, kRows * (count + 1) * sizeof(int64_t)), "prefix");
    if (st == FSI_OK) st = prec == FSI_F64 ? build_batch<double>(b) : build_batch<float>(b);
    if (st != FSI_OK) {
        fsi_batch_destroy(b);
        return st;
    }
    *out = b;
    return FSI_OK;
}

void fsi_batch_destroy(fsi_batch *b)
{
    if (!b) return;
    fsi::DeviceGuard _fsi_device_guard(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->desc_res);
    cudaFree(b->desc_jac);
    cudaFree(b->desc_dlm);
    cudaFree(b->prefix);
    cudaFree(b->blocks);
    cudaFree(b->spread);
    cudaFree(b->loc);
    cudaFree(b->xi64);
    delete b;
}

fsi_status fsi_batch_run(fsi_batch *b, int mode)
{
    if (!b) return set_error(FSI_ERR_ARG, "batch is NULL");
    if (mode < FSI_BATCH_PER_INSTANCE || mode > FSI_BATCH_GRAPH)
        return set_error(FSI_ERR_ARG, "bad batch mode %d", mode);
    FSI_DEVICE(b->device);
    return run_mode(b, mode, kAllPhases);
}

fsi_status fsi_batch_autotune(fsi_batch *b, int reps, fsi_tune_report *rep)
{
    if (!b || !rep || reps < 1) return set_error(FSI_ERR_ARG, "bad autotune arguments");
    FSI_DEVICE(b->device);
    std::memset(rep, 0, sizeof *rep);
    const Brick start = b->brick;
    const int start_ctas = b->ctas_per_sm;
    double best = 1e30;
    Brick best_brick = start;
    int best_ctas = start_ctas;
    int tried = 0;
    for (const Brick &cand : kBrickCandidates) {
        for (int ctas : {1, 2, 4, 8}) {
            b->brick = cand;
            b->ctas_per_sm = ctas;
            FSI_TRY(b->prec == FSI_F64 ? build_batch<double>(b) : build_batch<float>(b));
            double t = 0.0;
            FSI_TRY(time_mode(b, FSI_BATCH_PERSISTENT, 3, reps, &t));
            if (tried < FSI_TUNE_MAX_CANDIDATES) {
                rep->cand_bx[tried] = cand.bx;
                rep->cand_by[tried] = cand.by;
                rep->cand_bz[tried] = cand.bz;
                rep->cand_ctas[tried] = ctas;
                rep->cand_seconds[tried] = t;
            }
            ++tried;
            if (t < best) {
                best = t;
                best_brick = cand;
                best_ctas = ctas;
            }
        }
    }
    b->brick = best_brick;
    b->ctas_per_sm = best_ctas;
    FSI_TRY(b->prec == FSI_F64 ? build_batch<double>(b) : build_batch<float>(b));
    rep->n_candidates = tried < FSI_TUNE_MAX_CANDIDATES ? tried : FSI_TUNE_MAX_CANDIDATES;
    rep->bx = best_brick.bx;
    rep->by = best_brick.by;
    rep->bz = best_brick.bz;
    rep->threads = best_brick.threads;
    rep->ctas_per_sm = best_ctas;
    rep->seconds = best;
    // persist the choice (one JSON object per line) when FSI_TUNE_CACHE is set
    const char *path = getenv("FSI_TUNE_CACHE");
    if (path && *path) {
        FILE *f = fopen(path, "a");
        if (f) {
            fprintf(f,
                    "{\"kind\": \"batch\", \"instances\": %d, \"prec\": \"%s\", \"bx\": %d, "
                    "\"by\": %d, \"bz\": %d, \"threads\": %d, \"ctas_per_sm\": %d, "
                    "\"seconds\": %.6e}\n",
                    b->count, b->prec == FSI_F64 ? "f64" : "f32", best_brick.bx, best_brick.by,
                    best_brick.bz, best_brick.threads, best_ctas, best);
            fclose(f);
        }
    }
    return FSI_OK;
}

fsi_status fsi_batch_time(fsi_batch *b, int mode, int reps, double *seconds)
{
    if (!b || !seconds || reps < 1) return set_error(FSI_ERR_ARG, "bad arguments");
    if (mode < FSI_BATCH_PER_INSTANCE || mode > FSI_BATCH_GRAPH)
        return set_error(FSI_ERR_ARG, "bad batch mode %d", mode);
    FSI_DEVICE(b->device);
    return time_mode(b, mode, kAllPhases, reps, seconds);
}

}  // extern "C"
