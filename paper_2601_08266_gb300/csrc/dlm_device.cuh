// dlm_device.cuh -- per-work-item device code of the coupling operators,
// shared by the single-mesh kernels (dlm.cu) and the batched persistent
// kernels (batch.cu).  See dlm.cu for the design.
#pragma once

#include <cmath>
#include <cstring>

#include "df64.cuh"
#include "fsi_internal.cuh"

namespace fsi {
namespace dlmd {

struct GridArgs {
    int Nx, Ny, Nz;
    double x0, y0, z0, hx, hy, hz;
    // 1/h_k when h_k is an exact power of two (then d * (1/h_k) is the
    // correctly rounded d / h_k: both round the same real number d 2^-e), else 0
    double rx, ry, rz;
    // shifted: every 1/h_k = 2^s_k with 0 <= s_k <= 1000, and then the bit
    // patterns of d_max_k = N_k h_k (exact; see locate_point)
    int shifted;
    int sx, sy, sz;
    long long dmax_bits[3];
    int zero_origin;  // x0_k == 0 (either sign) on every axis
    // exact division of an element index e < 2^31 by Nx and by Ny:
    // e / N = (e * div_m) >> div_k (see division_magic)
    unsigned long long div_mx, div_my;
    int div_kx, div_ky;
};

// multiplier and shift of the exact division by d (1 <= d < 2^31) of every
// n < 2^31: k = 31 + ceil(log2 d), M = ceil(2^k / d); then M d - 2^k < d and
// n M / 2^k < n/d + 2^(31-k) <= n/d + 1/d, which cannot pass the next integer
inline void division_magic(int d, unsigned long long &M, int &k)
{
    int l = 0;
    while ((1LL << l) < d) ++l;
    k = 31 + l;
    M = ((1ULL << k) + (unsigned long long)d - 1) / (unsigned long long)d;
}

// the exact reciprocal of h when h = 2^e (with 1/h a normal double), else 0
inline double pow2_reciprocal(double h)
{
    int e = 0;
    const double f = std::frexp(h, &e);  // h = f 2^e, f in [0.5, 1)
    if (!(h > 0.0) || f != 0.5) return 0.0;
    const double r = std::ldexp(1.0, 1 - e);
    return (std::isnormal(r) && r * h == 1.0) ? r : 0.0;
}

inline void set_reciprocals(GridArgs &g)
{
    g.rx = pow2_reciprocal(g.hx);
    g.ry = pow2_reciprocal(g.hy);
    g.rz = pow2_reciprocal(g.hz);
    const double r[3] = {g.rx, g.ry, g.rz}, h[3] = {g.hx, g.hy, g.hz};
    const int N[3] = {g.Nx, g.Ny, g.Nz};
    int sh[3] = {0, 0, 0};
    g.shifted = 1;
    for (int k = 0; k < 3; ++k) {
        int e = 0;
        std::frexp(r[k], &e);  // r = 0.5 * 2^e = 2^(e-1) when r is a power of two
        sh[k] = e - 1;
        if (!(r[k] >= 1.0) || sh[k] > 1000) g.shifted = 0;
        const double dmax = (double)N[k] * h[k];  // exact: N < 2^31 times 2^-s
        std::memcpy(&g.dmax_bits[k], &dmax, sizeof dmax);
    }
    g.zero_origin = g.x0 == 0.0 && g.y0 == 0.0 && g.z0 == 0.0;
    division_magic(g.Nx, g.div_mx, g.div_kx);
    division_magic(g.Ny, g.div_my, g.div_ky);
    g.sx = sh[0];
    g.sy = sh[1];
    g.sz = sh[2];
}

// (X - x0) / h as IEEE FP64 division, by the exact multiply when h is a
// power of two (GB300's FP64 division is a long dependent sequence)
__device__ __forceinline__ double grid_coord(double X, double x0, double h, double r)
{
    const double d = X - x0;
    return r != 0.0 ? d * r : d / h;
}

// ------------------------------------------------------------ location
// Location of point b on the uniform grid: t_k = (X_k - x0_k)/h_k, outside
// unless 0 <= t_k <= N_k (NaN is outside), e_k = min(floor(t_k), N_k - 1),
// xi_k = 2 (t_k - e_k) - 1, all in FP64 (xi stored in S).  Writes elem[b]
// and xi[b]; returns the element, or -1 for an outside point (xi = 0).
//
// With every h_k = 2^-s_k (s_k >= 0), t_k = d_k 2^s_k is exact, so the same
// results follow from integer work on the bits of d_k = X_k - x0_k (GB300's
// FP64 unit issues two operations per SM and clock): 0 <= t_k <= N_k is 0 <=
// d_k <= N_k h_k (an exact double) compared as ordered bit patterns;
// floor(t_k) is the integer part of d_k's significand shifted by its
// exponent + s_k; for floor(t_k) >= 1, xi_k = 2 (t_k - e_k) - 1 is exactly
// Z 2^(u-52), u the exponent of t_k and Z = 2 F - 2^(52-u) (F the fraction
// bits of t_k, |Z| < 2^53); in the first cell (t_k < 1), 2 t_k - 1 is
// rounded to nearest, ties to even, from its exact integer form, as the FP64
// subtraction of the definition rounds it.  Only a non-zero origin costs an
// FP64 subtraction per coordinate.

// the double of a non-zero integer Z (|Z| <= 2^53) times 2^p, from its bits
// (the result is normal)
__host__ __device__ __forceinline__ double exact_scaled(long long Z, int p)
{
    const long long a = Z < 0 ? -Z : Z;
#ifdef __CUDA_ARCH__
    const int msb = 63 - __clzll(a);
#else
    const int msb = 63 - __builtin_clzll((unsigned long long)a);
#endif
    const long long b = ((long long)(Z < 0) << 63) | ((long long)(1023 + msb + p) << 52) |
                        ((a << (52 - msb)) & 0xfffffffffffffLL);
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double r;
    std::memcpy(&r, &b, sizeof r);
    return r;
#endif
}

// 2 t - 1 rounded to nearest (ties to even) for t = d 2^s in [0, 1), from
// the bits of d (d >= 0 or -0; s <= 1000)
__host__ __device__ __forceinline__ double first_cell_xi(long long bits, int s)
{
    const int be = (int)((bits >> 52) & 0x7ff);
    long long sig = bits & 0xfffffffffffffLL;
    int u;  // t = sig 2^(u - 52)
    if (be == 0) {
        u = -1022 + s;
    } else {
        sig |= 1LL << 52;
        u = be - 1023 + s;
    }
    if (sig == 0) return -1.0;
    if (be != 0 && u == -1) {  // t in [1/2, 1): 2t - 1 = (sig - 2^52) 2^-52, exact
        const long long Z = sig - (1LL << 52);
        return Z == 0 ? 0.0 : exact_scaled(Z, -52);
    }
    // t < 1/2: 2t - 1 = -(2^53 - y) 2^-53, y = sig 2^(u+2) = sig / 2^j < 2^52
    const int j = -u - 2;
    long long M;
    if (j <= 0) {
        M = (1LL << 53) - (sig << (-j));
    } else if (j >= 60) {
        M = 1LL << 53;  // y < 2^-7
    } else {
        const long long q = sig >> j, r = sig & ((1LL << j) - 1), half = 1LL << (j - 1);
        const long long B = (1LL << 53) - q, A = B - 1;  // 2^53 - y lies in (A, B]
        M = r == 0 ? B : (r < half ? B : (r > half ? A : ((B & 1) ? A : B)));
    }
    return M == (1LL << 53) ? -1.0 : exact_scaled(-M, -53);
}

// axis k of the shifted path: returns false when the point is outside on it
template <bool ZERO_ORIGIN>
__device__ __forceinline__ bool shifted_axis(double X, double x0, int s, long long dmax_bits,
                                             int N, int &e, double &q)
{
    const double d = ZERO_ORIGIN ? X : X - x0;  // X - (+-0) is X up to the sign of a zero
    const long long bits = __double_as_longlong(d);
    if (!(bits <= dmax_bits && (bits >= 0 || bits == (long long)0x8000000000000000ULL)))
        return false;
    const int be = (int)((bits >> 52) & 0x7ff);  // biased exponent of d
    const int u = be - 1023 + s;                 // exponent of t = d 2^s
    if (be == 0 || u < 0) {                      // t < 1
        e = 0;
        q = first_cell_xi(bits, s);
        return true;
    }
    const long long sig = (bits & 0xfffffffffffffLL) | (1LL << 52);
    const int f = (int)(sig >> (52 - u));  // floor(t) >= 1, u <= 30
    if (f >= N) {                          // t = N: the last cell's far face
        e = N - 1;
        q = 1.0;
        return true;
    }
    e = f;
    const long long Z = 2 * (sig & ((1LL << (52 - u)) - 1)) - (1LL << (52 - u));
    q = Z == 0 ? 0.0 : exact_scaled(Z, u - 52);
    return true;
}

// ZERO_ORIGIN: the caller has checked g.zero_origin (x0 = 0 on every axis)
template <typename S, bool ZERO_ORIGIN = false>
__device__ __forceinline__ int locate_point(const GridArgs &g, int64_t b,
                                            const double *__restrict__ X,
                                            int32_t *__restrict__ elem, S *__restrict__ xi)
{
    if (g.shifted) {
        int ex = 0, ey = 0, ez = 0;
        double qx = 0.0, qy = 0.0, qz = 0.0;
        const bool in =
            shifted_axis<ZERO_ORIGIN>(X[3 * b + 0], g.x0, g.sx, g.dmax_bits[0], g.Nx, ex, qx) &
            shifted_axis<ZERO_ORIGIN>(X[3 * b + 1], g.y0, g.sy, g.dmax_bits[1], g.Ny, ey, qy) &
            shifted_axis<ZERO_ORIGIN>(X[3 * b + 2], g.z0, g.sz, g.dmax_bits[2], g.Nz, ez, qz);
        if (!in) {
            elem[b] = -1;
            xi[3 * b + 0] = S(0);
            xi[3 * b + 1] = S(0);
            xi[3 * b + 2] = S(0);
            return -1;
        }
        xi[3 * b + 0] = (S)qx;
        xi[3 * b + 1] = (S)qy;
        xi[3 * b + 2] = (S)qz;
        const int e = ex + g.Nx * (ey + g.Ny * ez);
        elem[b] = e;
        return e;
    }
    const double tx = grid_coord(X[3 * b + 0], g.x0, g.hx, g.rx);
    const double ty = grid_coord(X[3 * b + 1], g.y0, g.hy, g.ry);
    const double tz = grid_coord(X[3 * b + 2], g.z0, g.hz, g.rz);
    const bool in = (tx >= 0.0 && tx <= (double)g.Nx) && (ty >= 0.0 && ty <= (double)g.Ny) &&
                    (tz >= 0.0 && tz <= (double)g.Nz);
    if (!in) {
        elem[b] = -1;
        xi[3 * b + 0] = S(0);
        xi[3 * b + 1] = S(0);
        xi[3 * b + 2] = S(0);
        return -1;
    }
    const int ex = min((int)floor(tx), g.Nx - 1);
    const int ey = min((int)floor(ty), g.Ny - 1);
    const int ez = min((int)floor(tz), g.Nz - 1);
    xi[3 * b + 0] = (S)(2.0 * (tx - (double)ex) - 1.0);
    xi[3 * b + 1] = (S)(2.0 * (ty - (double)ey) - 1.0);
    xi[3 * b + 2] = (S)(2.0 * (tz - (double)ez) - 1.0);
    const int e = ex + g.Nx * (ey + g.Ny * ez);
    elem[b] = e;
    return e;
}

// ------------------------------------------------------------ cell table
// Exclusive scan of count[0..E) into start[0..E] (start[E] = total) with
// 2048-entry tiles: (1) tile-local inclusive scan + tile totals, (2) one CTA
// scans the tile totals, (3) tiles add their offset.  The bodies below take
// one tile (1024 threads) or the CTA of step (2).
constexpr int kScanTile = 2048;

// scan tiles of a table of E cells
__host__ __device__ inline int64_t cell_tiles(int64_t E) { return (E + kScanTile - 1) / kScanTile; }

__device__ __forceinline__ int block_inclusive_scan(int v, int *warp_sums)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    if (wid > 0) v += warp_sums[wid - 1];
    return v;
}

__device__ __forceinline__ void scan_tile(int64_t E, const int32_t *count, int32_t *start,
                                          int32_t *tile_sum, int64_t tile, int *warp_sums)
{
    const int64_t base = tile * kScanTile + 2 * threadIdx.x;
    const int a = base < E ? count[base] : 0;
    const int b = base + 1 < E ? count[base + 1] : 0;
    const int incl = block_inclusive_scan(a + b, warp_sums);
    if (base < E) start[base + 1] = incl - b;
    if (base + 1 < E) start[base + 2] = incl;
    if (threadIdx.x == blockDim.x - 1) tile_sum[tile] = incl;
}

__device__ __forceinline__ void scan_totals_block(int64_t ntiles, int32_t *tile_sum,
                                                  int *warp_sums, int *carry)
{
    if (threadIdx.x == 0) *carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int v = i < ntiles ? tile_sum[i] : 0;
        const int incl = block_inclusive_scan(v, warp_sums);
        const int c = *carry;
        __syncthreads();
        if (i < ntiles) tile_sum[i] = c + incl - v;  // exclusive
        if (threadIdx.x == blockDim.x - 1) *carry = c + incl;
        __syncthreads();
    }
}

__device__ __forceinline__ void scan_add_tile(int64_t E, int32_t *start, const int32_t *tile_sum,
                                              int64_t tile)
{
    const int64_t base = tile * kScanTile;
    const int off = tile_sum[tile];
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        const int64_t k = base + i;
        if (k < E) start[k + 1] += off;
    }
    if (tile == 0 && threadIdx.x == 0) start[0] = 0;
}

// Sorting a cell's slice of perm ascending (restores the stable order; cell
// E is the tail of outside points [start[E], m)): one lane's shell sort, the
// fallback for slices too long for a CTA's shared memory.
__device__ inline void shell_sort(int32_t *s, int len)
{
    int gap = 1;
    while (gap * 9 / 4 + 1 < len) gap = gap * 9 / 4 + 1;
    for (;;) {
        for (int i = gap; i < len; ++i) {
            const int v = s[i];
            int j = i;
            while (j >= gap && s[j - gap] > v) {
                s[j] = s[j - gap];
                j -= gap;
            }
            s[j] = v;
        }
        if (gap == 1) break;
        gap = gap * 4 / 9;
        if (gap < 1) gap = 1;
    }
}

// Slices of up to kWarpSortMax points are ordered by a warp (the in-place
// table) or the rank pass (the single-mesh table with point scratch); fuller
// cells are listed and sorted by a whole CTA in shared memory
// (block_sort_cell), up to kBlockSortMax points, beyond which one lane
// shell-sorts the slice.
constexpr int kWarpSortMax = 128;
constexpr int kBlockSortMax = 32768;

// Sort the slice of cell c (cell E: the outside points) with the whole CTA: a
// bitonic network over the slice padded with INT32_MAX to a power of two, in
// shared memory sh (kBlockSortMax ints).  Every thread of the CTA calls it.
__device__ __forceinline__ void block_sort_cell(int64_t E, int64_t m,
                                                const int32_t *__restrict__ start,
                                                int32_t *__restrict__ perm, int64_t c, int32_t *sh)
{
    const int lo = start[c];
    const int len = (c < E ? start[c + 1] : (int)m) - lo;
    if (len > kBlockSortMax) {
        if (threadIdx.x == 0) shell_sort(perm + lo, len);
        __syncthreads();
        return;
    }
    int P = 1;
    while (P < len) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < len ? perm[lo + i] : INT32_MAX;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const int a = sh[i], b = sh[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        sh[i] = b;
                        sh[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < len; i += blockDim.x) perm[lo + i] = sh[i];
    __syncthreads();
}

// (ex, ey, ez) of element e = ex + Nx (ey + Ny ez), 0 <= e < 2^31
__device__ __forceinline__ void elem_coords(const GridArgs &g, int e, int &ex, int &ey, int &ez)
{
    const int q = (int)(((unsigned long long)e * g.div_mx) >> g.div_kx);  // e / Nx
    ez = (int)(((unsigned long long)q * g.div_my) >> g.div_ky);          // q / Ny
    ex = e - q * g.Nx;
    ey = q - ez * g.Ny;
}

template <typename T> __device__ __forceinline__ T shape_1d(T xi, int side)
{
    return side ? (T(1) + xi) : (T(1) - xi);
}

// Interpolation for one point b (u = C^T V, Eq. nodal_solid_velo) by one
// lane (the double-float and FP64 kernels: issue-bound, so no work is
// duplicated).  T is the compute type; xi, U and u are in StorageOf<T>.
template <typename T>
__device__ __forceinline__ void interp_point(
    const GridArgs &g, int64_t b, const int32_t *__restrict__ elem,
    const typename StorageOf<T>::type *__restrict__ xi,
    const vec4<typename StorageOf<T>::type> *__restrict__ U,
    typename StorageOf<T>::type *__restrict__ u)
{
    const int NX1 = g.Nx + 1, NXY1 = (g.Nx + 1) * (g.Ny + 1);
    const int E = g.Nx * g.Ny * g.Nz;
    const int e = elem[b];
    T ux = T(0), uy = T(0), uz = T(0);
    if (e >= 0 && e < E) {
        int ex, ey, ez;
        elem_coords(g, e, ex, ey, ez);
        const T x0 = to_c<T>(xi[3 * b]), x1 = to_c<T>(xi[3 * b + 1]),
                x2 = to_c<T>(xi[3 * b + 2]);
        const int n0 = ex + NX1 * ey + NXY1 * ez;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
            const T Na = shape_1d(x0, ax) * shape_1d(x1, ay) * shape_1d(x2, az) * T(0.125f);
            const auto v = ld4(U + n0 + ax + NX1 * ay + NXY1 * az);
            ux = madd(Na, to_c<T>(v.x), ux);
            uy = madd(Na, to_c<T>(v.y), uy);
            uz = madd(Na, to_c<T>(v.z), uz);
        }
    }
    u[3 * b] = to_s(ux);
    u[3 * b + 1] = to_s(uy);
    u[3 * b + 2] = to_s(uz);
}

// The same by two adjacent lanes of a warp (the FP32 kernels: bound by the
// number of memory lines their node loads touch): lane ax (= lane & 1) sums the 4 nodes of the
// element with x-offset ax (in a = 2 (ay + 2 az) + ax order), so that the two
// lanes' loads of an x-adjacent node pair fall in one memory line; the ax = 0
// lane adds the other half and writes u.  Every lane of the warp calls this
// (valid == false: no point, no memory access), because of the shuffle.  T
// is the compute type; xi, U and u are in StorageOf<T>.
template <typename T>
__device__ __forceinline__ void interp_point_pair(
    const GridArgs &g, int64_t b, bool valid, const int32_t *__restrict__ elem,
    const typename StorageOf<T>::type *__restrict__ xi,
    const vec4<typename StorageOf<T>::type> *__restrict__ U,
    typename StorageOf<T>::type *__restrict__ u)
{
    const int NX1 = g.Nx + 1, NXY1 = (g.Nx + 1) * (g.Ny + 1);
    const int E = g.Nx * g.Ny * g.Nz;
    const int ax = threadIdx.x & 1;
    const int e = valid ? elem[b] : -1;
    T ux = T(0), uy = T(0), uz = T(0);
    if (e >= 0 && e < E) {
        int ex, ey, ez;
        elem_coords(g, e, ex, ey, ez);
        const T x0 = to_c<T>(xi[3 * b]), x1 = to_c<T>(xi[3 * b + 1]),
                x2 = to_c<T>(xi[3 * b + 2]);
        const int n0 = ex + ax + NX1 * ey + NXY1 * ez;
        const T sx = shape_1d(x0, ax);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ay = q & 1, az = q >> 1;
            const T Na = sx * shape_1d(x1, ay) * shape_1d(x2, az) * T(0.125f);
            const auto v = ld4(U + n0 + NX1 * ay + NXY1 * az);
            ux = madd(Na, to_c<T>(v.x), ux);
            uy = madd(Na, to_c<T>(v.y), uy);
            uz = madd(Na, to_c<T>(v.z), uz);
        }
    }
    ux = ux + shfl_x(ux, 1);
    uy = uy + shfl_x(uy, 1);
    uz = uz + shfl_x(uz, 1);
    if (valid && ax == 0) {
        u[3 * b] = to_s(ux);
        u[3 * b + 1] = to_s(uy);
        u[3 * b + 2] = to_s(uz);
    }
}

// Corner contributions w_B N_a(xi_B) lambda_B of one point B added to acc
// (T the compute type; inputs in StorageOf<T>).  SQ: w_B N_a(xi_B)^2 dsq
// instead (lam unused): the diagonal of C W C^T scaled by dsq.
template <typename T, bool SQ = false>
__device__ __forceinline__ void spread_accumulate(
    int b, const typename StorageOf<T>::type *__restrict__ xi,
    const typename StorageOf<T>::type *__restrict__ lam,
    const typename StorageOf<T>::type *__restrict__ w, T (&acc)[24], T dsq = T(0))
{
    const T x0 = to_c<T>(xi[3 * b]), x1 = to_c<T>(xi[3 * b + 1]), x2 = to_c<T>(xi[3 * b + 2]);
    const T s = w ? to_c<T>(w[b]) * T(0.125f) : T(0.125f);
    T l0, l1, l2;
    if constexpr (SQ) {
        l0 = l1 = l2 = dsq;
    } else {
        l0 = to_c<T>(lam[3 * b]);
        l1 = to_c<T>(lam[3 * b + 1]);
        l2 = to_c<T>(lam[3 * b + 2]);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const T sh = shape_1d(x0, a & 1) * shape_1d(x1, (a >> 1) & 1) * shape_1d(x2, (a >> 2) & 1);
        // N_a = sh / 8: w N_a = sh s, w N_a^2 = sh s (sh / 8)
        const T Na = SQ ? sh * s * (sh * T(0.125f)) : sh * s;
        acc[3 * a] = madd(Na, l0, acc[3 * a]);
        acc[3 * a + 1] = madd(Na, l1, acc[3 * a + 1]);
        acc[3 * a + 2] = madd(Na, l2, acc[3 * a + 2]);
    }
}

// Spreading, pass 1, on one segment of kSpreadSeg = 8 consecutive cells
// (called by all 32 lanes of a warp for the cells [c0, c0 + 8)).  Four lanes
// share a cell of at most kGroupCell points: lane k of the group sums the
// cell's points k, k+4, ... (perm order) into the 8 corner contributions
// w_B N_a(xi_B) lambda_B (24 values), then a two-level transpose-reduce over
// the group leaves 6 corner sums in each lane.  Fuller cells are taken by the
// whole warp: the lanes stride over the points and a five-level
// transpose-reduce gives the sums.  Every cell's corner sums S[cell][8][3]
// come out of a fixed order of operations, so the result is deterministic.
// (Thin leaflets occupy few cells of few rows: short segments spread them
// over more warps.)
constexpr int kSpreadSeg = 8;
constexpr int kGroupCell = 128;

template <typename T, bool SQ = false>
__device__ __forceinline__ void spread_cells_segment(
    int64_t E, int64_t c0, const typename StorageOf<T>::type *__restrict__ xi,
    const int32_t *__restrict__ start, const int32_t *__restrict__ perm,
    const typename StorageOf<T>::type *__restrict__ lam,
    const typename StorageOf<T>::type *__restrict__ w, T *__restrict__ S, T dsq = T(0))
{
    const int lane = threadIdx.x & 31;
    const int64_t myc = c0 + (lane >> 2);
    int lo = 0, hi = 0;
    if (myc < E) {
        lo = start[myc];
        hi = start[myc + 1];
    }
    if (__all_sync(0xffffffffu, hi == lo)) return;
    {
        const bool group = hi - lo <= kGroupCell;
        T acc[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] = T(0);
        if (group)
            for (int p = lo + (lane & 3); p < hi; p += 4) spread_accumulate<T, SQ>(perm[p], xi, lam, w, acc, dsq);
        const bool b1 = lane & 2, b0 = lane & 1;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const T send = b1 ? acc[k] : acc[12 + k];
            const T keep = b1 ? acc[12 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 2);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const T send = b0 ? acc[k] : acc[6 + k];
            const T keep = b0 ? acc[6 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 1);
        }
        if (group && hi > lo) {
            T *dst = S + myc * 24 + (b1 ? 12 : 0) + (b0 ? 6 : 0);
#pragma unroll
            for (int k = 0; k < 6; ++k) dst[k] = acc[k];
        }
    }
    // fuller cells: the whole warp, one cell after the other
    unsigned occ = __ballot_sync(0xffffffffu, hi - lo > kGroupCell && (lane & 3) == 0);
    while (occ) {
        const int l = __ffs(occ) - 1;
        occ &= occ - 1;
        const int plo = __shfl_sync(0xffffffffu, lo, l);
        const int phi = __shfl_sync(0xffffffffu, hi, l);
        T acc[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] = T(0);
        for (int p = plo + lane; p < phi; p += 32) spread_accumulate<T, SQ>(perm[p], xi, lam, w, acc, dsq);
        // each level halves the values a lane carries (12, 6, 3), then a
        // butterfly over the last two bits
        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const T send = b4 ? acc[k] : acc[12 + k];
            const T keep = b4 ? acc[12 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 16);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const T send = b3 ? acc[k] : acc[6 + k];
            const T keep = b3 ? acc[6 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 8);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T send = b2 ? acc[k] : acc[3 + k];
            const T keep = b2 ? acc[3 + k] : acc[k];
            acc[k] = keep + shfl_x(send, 4);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            acc[k] = acc[k] + shfl_x(acc[k], 2);
            acc[k] = acc[k] + shfl_x(acc[k], 1);
        }
        if ((lane & 3) == 0) {
            const int idx0 = (b4 ? 12 : 0) + (b3 ? 6 : 0) + (b2 ? 3 : 0);
            T *dst = S + (c0 + (l >> 2)) * 24 + idx0;
            dst[0] = acc[0];
            dst[1] = acc[1];
            dst[2] = acc[2];
        }
    }
}

// Spreading, pass 2: node (i, j, k) sums the corner sums of its (up to 8)
// occupied cells in a fixed order (c = 0..7, cx fastest).  The node is
// corner (cx, cy, cz) of cell (i - cx, j - cy, k - cz); the two cells of a
// row pair (i - 1, i) are tested with three cell-table entries.
template <typename T>
__device__ __forceinline__ void spread_node(const GridArgs &g, int i, int j, int k,
                                            const int32_t *__restrict__ start,
                                            const T *__restrict__ S,
                                            typename StorageOf<T>::type *__restrict__ F,
                                            int accumulate)
{
    using St = typename StorageOf<T>::type;
    St *o = F + 4 * ((size_t)i + (size_t)(g.Nx + 1) * (j + (size_t)(g.Ny + 1) * k));
    // the (up to) four rows of cells around the node; a row without points
    // (most rows, for thin leaflets) is told by two entries that every node
    // of the row reads alike, and a node with no such row is done at once
    // (a branch the lanes of a warp, one node row, take alike)
    const int32_t *row[4];
    bool rocc[4];
#pragma unroll
    for (int rc = 0; rc < 4; ++rc) {
        const int ey = j - (rc & 1), ez = k - (rc >> 1);
        rocc[rc] = false;
        row[rc] = start;
        if (ey < 0 || ez < 0 || ey >= g.Ny || ez >= g.Nz) continue;
        row[rc] = start + (size_t)g.Nx * (ey + (size_t)g.Ny * ez);
        rocc[rc] = row[rc][g.Nx] != row[rc][0];
    }
    if (!(rocc[0] | rocc[1] | rocc[2] | rocc[3])) {
        if (!accumulate) {
            o[0] = St(0);
            o[1] = St(0);
            o[2] = St(0);
        }
        return;
    }
    bool occ[8];
#pragma unroll
    for (int rc = 0; rc < 4; ++rc) {
        occ[2 * rc] = occ[2 * rc + 1] = false;
        if (!rocc[rc]) continue;
        // st[0] = start of cell i of the row (for i = Nx the entry after the
        // row's last cell, still inside the table's E + 1 entries)
        const int32_t *st = row[rc] + i;
        const int s0 = st[0];
        if (i < g.Nx) occ[2 * rc] = st[1] > s0;      // cell i     (cx = 0)
        if (i > 0) occ[2 * rc + 1] = s0 > st[-1];    // cell i - 1 (cx = 1)
    }
    T fx = T(0), fy = T(0), fz = T(0);
    bool touched = false;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (!occ[c]) continue;
        const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        const int cell = (i - cx) + g.Nx * ((j - cy) + g.Ny * (k - cz));
        const T *sc = S + (size_t)cell * 24 + 3 * c;
        fx = fx + sc[0];
        fy = fy + sc[1];
        fz = fz + sc[2];
        touched = true;
    }
    if (accumulate) {
        if (touched) {
            o[0] = to_s(to_c<T>(o[0]) + fx);
            o[1] = to_s(to_c<T>(o[1]) + fy);
            o[2] = to_s(to_c<T>(o[2]) + fz);
        }
    } else {
        o[0] = to_s(fx);
        o[1] = to_s(fy);
        o[2] = to_s(fz);
    }
}

}  // namespace dlmd
}  // namespace fsi
