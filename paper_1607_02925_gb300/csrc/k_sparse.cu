// Sparse X (d x n, FP32 values) on the device: validation of the caller's CSR
// of the rows of X, the compressed columns x_i built from it (a stable
// transpose: counting sort by column, then each column sorted by row), the
// row work list of the X Y product, and the kernels of the anchor pass
// (Sec. 2.3: Y = X^T W over the columns, G = X Y over the rows), of the column
// norms (a0) and of the SVRG inner loop in factored form.
//
// Every reduction runs in a fixed order, so results do not depend on timing:
// the transpose's atomic cursor only decides where an entry lands before its
// column is sorted by (unique) row index.
#include <algorithm>
#include <type_traits>

#include "kernels.cuh"

namespace lra {

namespace {

constexpr int kWarps = 8;  // warps per CTA of the warp-per-row/column kernels

__device__ __forceinline__ int64_t global_warp() {
    return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}
__device__ __forceinline__ int64_t warps_in_grid() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

unsigned grid_for(int64_t items, int per_block) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(items, per_block), 152 * 16));
}

// ---------------------------------------------------------------------------
// Validation: bit 1 row pointer out of order or range, 2 column index out of
// [0, n), 4 column indices not strictly increasing within a row, 8 a value
// not finite, 16 rowptr[0] != 0 or rowptr[d] != nnz.
// ---------------------------------------------------------------------------
__global__ void csr_check_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                 const float *__restrict__ val, int64_t d, int64_t n, int64_t nnz,
                                 int *__restrict__ bad) {
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rowptr[0] != 0 || rowptr[d] != nnz) atomicOr(bad, 16);
    }
    int flags = 0;
    for (int64_t r = global_warp(); r < d; r += warps_in_grid()) {
        const int64_t lo = rowptr[r], hi = rowptr[r + 1];
        if (lo < 0 || hi < lo || hi > nnz) {
            flags |= 1;
            continue;
        }
        for (int64_t k = lo + lane; k < hi; k += 32) {
            const int32_t c = colidx[k];
            if (c < 0 || (int64_t)c >= n) flags |= 2;
            if (k + 1 < hi && colidx[k + 1] <= c) flags |= 4;
            if (!isfinite(val[k])) flags |= 8;
        }
    }
    if (flags) atomicOr(bad, flags);
}

// ---------------------------------------------------------------------------
// Exclusive scan of int64 counts: out[0] = 0, out[i + 1] = in[0] + ... + in[i].
// Tiles of 1024 (one element per thread), tile totals scanned by one CTA.
// ---------------------------------------------------------------------------
constexpr int kScanTile = 1024;

__device__ int64_t block_incl_scan(int64_t v, int64_t *warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        warp_tot[lane] = s;
    }
    __syncthreads();
    if (w > 0) v += warp_tot[w - 1];
    return v;
}

__global__ void __launch_bounds__(kScanTile) scan_tiles_kernel(const int64_t *__restrict__ in, int64_t N,
                                                               int64_t *__restrict__ out,
                                                               int64_t *__restrict__ tile_tot) {
    __shared__ int64_t wt[32];
    const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    const int64_t v = block_incl_scan(i < N ? in[i] : 0, wt);
    if (i < N) out[i + 1] = v;
    if (threadIdx.x == kScanTile - 1) tile_tot[blockIdx.x] = v;
}

// one CTA: exclusive scan of the tile totals, in chunks of 1024 with a carry
__global__ void __launch_bounds__(kScanTile) scan_totals_kernel(int64_t *__restrict__ tile_tot, int64_t T) {
    __shared__ int64_t wt[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < T; base += kScanTile) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < T ? tile_tot[i] : 0;
        const int64_t incl = block_incl_scan(v, wt);
        const int64_t c = carry;
        if (i < T) tile_tot[i] = c + incl - v;  // exclusive
        __syncthreads();
        if (threadIdx.x == kScanTile - 1) carry = c + incl;
        __syncthreads();
    }
}

__global__ void scan_add_kernel(int64_t *__restrict__ out, int64_t N, const int64_t *__restrict__ tile_off) {
    const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    if (i < N) out[i + 1] += tile_off[blockIdx.x];
    if (i == 0) out[0] = 0;
}

// scratch >= ceil(N / 1024) int64
void exclusive_scan(cudaStream_t s, const int64_t *in, int64_t N, int64_t *out, int64_t *scratch) {
    const int64_t T = std::max<int64_t>(1, ceil_div(N, kScanTile));
    scan_tiles_kernel<<<(unsigned)T, kScanTile, 0, s>>>(in, N, out, scratch);
    LRA_LAUNCHED();
    scan_totals_kernel<<<1, kScanTile, 0, s>>>(scratch, T);
    LRA_LAUNCHED();
    scan_add_kernel<<<(unsigned)T, kScanTile, 0, s>>>(out, N, scratch);
    LRA_LAUNCHED();
}

// ---------------------------------------------------------------------------
// Transpose: column counts, scatter through per-column cursors, column sort.
// ---------------------------------------------------------------------------
__global__ void col_count_kernel(const int32_t *__restrict__ colidx, int64_t nnz,
                                 unsigned long long *__restrict__ cnt) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[colidx[k]], 1ull);
}

__global__ void col_scatter_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                   const float *__restrict__ val, int64_t d,
                                   const int64_t *__restrict__ colptr, int *__restrict__ cursor,
                                   int32_t *__restrict__ rowidx, float *__restrict__ cval) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = global_warp(); r < d; r += warps_in_grid()) {
        const int64_t lo = rowptr[r], hi = rowptr[r + 1];
        for (int64_t k = lo + lane; k < hi; k += 32) {
            const int32_t c = colidx[k];
            const int64_t pos = colptr[c] + atomicAdd(&cursor[c], 1);
            rowidx[pos] = (int32_t)r;
            cval[pos] = val[k];
        }
    }
}

// Ascending sort network for any length L (all comparators put the smaller key
// at the lower index; positions >= L act as +infinity and are never touched):
// for size = 2, 4, ... : compare i with its mirror in the size-block, then
// i with i + h for h = size/4, ..., 1.  `step(i, j)` is called for i < j < L.
template <bool kBlock>
__device__ __forceinline__ void net_sync() {
    if (kBlock)
        __syncthreads();
    else
        __syncwarp();
}

template <bool kBlock, typename F>
__device__ __forceinline__ void sort_network(int64_t L, int tid, int nthr, F &&step) {
    int64_t N = 1;
    while (N < L) N <<= 1;
    for (int64_t size = 2; size <= N; size <<= 1) {
        const int64_t half = size >> 1;
        for (int64_t t = tid; t < (N >> 1); t += nthr) {
            const int64_t blk = t / half, off = t - blk * half;
            const int64_t i = blk * size + off, j = blk * size + size - 1 - off;
            if (j < L) step(i, j);
        }
        net_sync<kBlock>();
        for (int64_t h = half >> 1; h > 0; h >>= 1) {
            for (int64_t t = tid; t < (N >> 1); t += nthr) {
                const int64_t i = (t / h) * 2 * h + (t % h), j = i + h;
                if (j < L) step(i, j);
            }
            net_sync<kBlock>();
        }
    }
}

constexpr int kSortWarp = 1024;  // longest column sorted by one warp in shared memory
constexpr int kSortWarps = 4;

__global__ void __launch_bounds__(32 * kSortWarps) sort_cols_warp_kernel(const int64_t *__restrict__ colptr,
                                                                        int64_t n, int32_t *__restrict__ rowidx,
                                                                        float *__restrict__ cval) {
    __shared__ int32_t ks[kSortWarps][kSortWarp];
    __shared__ float vs[kSortWarps][kSortWarp];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *K = ks[w];
    float *V = vs[w];
    for (int64_t c = global_warp(); c < n; c += warps_in_grid()) {
        const int64_t lo = colptr[c], L = colptr[c + 1] - lo;
        if (L < 2 || L > kSortWarp) continue;
        for (int64_t e = lane; e < L; e += 32) {
            K[e] = rowidx[lo + e];
            V[e] = cval[lo + e];
        }
        __syncwarp();
        auto step = [&](int64_t i, int64_t j) {
            if (K[i] > K[j]) {
                const int32_t tk = K[i];
                K[i] = K[j];
                K[j] = tk;
                const float tv = V[i];
                V[i] = V[j];
                V[j] = tv;
            }
        };
        sort_network<false>(L, lane, 32, step);
        for (int64_t e = lane; e < L; e += 32) {
            rowidx[lo + e] = K[e];
            cval[lo + e] = V[e];
        }
        __syncwarp();
    }
}

// columns longer than kSortWarp: one CTA per column, in place in global memory
__global__ void __launch_bounds__(512) sort_cols_block_kernel(const int64_t *__restrict__ colptr, int64_t n,
                                                              int32_t *__restrict__ rowidx,
                                                              float *__restrict__ cval) {
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
        const int64_t lo = colptr[c], L = colptr[c + 1] - lo;
        if (L <= kSortWarp) continue;
        int32_t *K = rowidx + lo;
        float *V = cval + lo;
        auto step = [&](int64_t i, int64_t j) {
            const int32_t ki = K[i], kj = K[j];
            if (ki > kj) {
                K[i] = kj;
                K[j] = ki;
                const float tv = V[i];
                V[i] = V[j];
                V[j] = tv;
            }
        };
        sort_network<true>(L, threadIdx.x, blockDim.x, step);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Row work list of X Y: row r of X is cut into ceil(len/seg) segments (one for
// empty rows and the padding rows d..dpad-1); item j = (row, segment).
// ---------------------------------------------------------------------------
__global__ void row_segs_kernel(const int64_t *__restrict__ rowptr, int64_t d, int64_t dpad, int seg,
                                int64_t *__restrict__ nseg) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dpad; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = 1;
        if (r < d) {
            s = ceil_div(rowptr[r + 1] - rowptr[r], seg);
            if (s < 1) s = 1;
        }
        nseg[r] = s;
    }
}

__global__ void fill_items_kernel(const int64_t *__restrict__ item_off, int64_t dpad, int2 *__restrict__ items) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dpad; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = item_off[r], e = item_off[r + 1];
        for (int64_t j = o; j < e; ++j) items[j] = make_int2((int)r, (int)(j - o));
    }
}

// ---------------------------------------------------------------------------
// Column norms ||x_i||^2 in FP64 (warp per column, fixed order)
// ---------------------------------------------------------------------------
__global__ void sparse_colnorms_kernel(const int64_t *__restrict__ colptr, const float *__restrict__ cval,
                                       int64_t n, double *__restrict__ norm2) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = global_warp(); i < n; i += warps_in_grid()) {
        double acc = 0.0;
        for (int64_t k = colptr[i] + lane; k < colptr[i + 1]; k += 32) {
            const double v = cval[k];
            acc = fma(v, v, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) norm2[i] = acc;
    }
}

// long rows: G[r] = sum of its segments in order
__global__ void __launch_bounds__(32 * kWarps) long_rows_kernel(const int64_t *__restrict__ item_off, int64_t dpad,
                                                                const float *__restrict__ partial, int PP,
                                                                float *__restrict__ G) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = global_warp(); r < dpad; r += warps_in_grid()) {
        const int64_t o = item_off[r], e = item_off[r + 1];
        if (e - o < 2) continue;
        for (int j = lane; j < PP; j += 32) {
            float a = 0.0f;
            for (int64_t t = o; t < e; ++t) a += partial[t * PP + j];
            G[r * PP + j] = a;
        }
    }
}

// ---------------------------------------------------------------------------
// Gather-accumulate with power-of-two lane groups (the X Y pass): GL lanes (4 GL >= p)
// take one entry, each lane a float4 of the gathered row, so 32 / GL entries
// are in flight per warp instruction; entries lo + g, lo + g + 32/GL, ... go
// to group g.  Rows below H come from the shared-memory copy `hot` (row
// stride p4 = p rounded up to 4); the others from B (row-major, PP wide)
// through the read-only path.  On return every lane holds the sum over the
// groups of its four columns (butterfly over the group bits: fixed order).
// ---------------------------------------------------------------------------
template <int GL>
__device__ __forceinline__ float4 gather_line4(const int32_t *__restrict__ idx, const float *__restrict__ vals,
                                               int64_t lo, int64_t hi, const float *__restrict__ B, int PP, int p,
                                               const float *hot, int H, int p4, int lane) {
    constexpr int NG = 32 / GL;
    const int g = lane / GL, l = lane % GL;
    const bool colok = 4 * l < p;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    // the (index, value) chunk of 32 entries is loaded one chunk ahead, with the
    // streaming (evict-first) hint: each entry is read once per pass, and the
    // gathered rows of B should keep the L2 lines
    int32_t rn = lo + lane < hi ? __ldcs(idx + lo + lane) : 0;
    float vn = lo + lane < hi ? __ldcs(vals + lo + lane) : 0.0f;
    for (int64_t base = lo; base < hi; base += 32) {
        const int32_t rr = rn;
        const float vv = vn;
        const int64_t k = base + 32 + lane;
        rn = k < hi ? __ldcs(idx + k) : 0;
        vn = k < hi ? __ldcs(vals + k) : 0.0f;
        const int cnt = (int)((hi - base) < 32 ? (hi - base) : 32);
#pragma unroll 4
        for (int e = 0; e < cnt; e += NG) {
            const int src = e + g;
            const int r = __shfl_sync(0xffffffffu, rr, src);
            const float v = __shfl_sync(0xffffffffu, vv, src);
            if (src < cnt && colok) {
                float4 b;
                if (r < H)
                    b = *reinterpret_cast<const float4 *>(hot + (int64_t)r * p4 + 4 * l);
                else
                    b = __ldg(reinterpret_cast<const float4 *>(B + (int64_t)r * PP + 4 * l));
                acc.x = fmaf(v, b.x, acc.x);
                acc.y = fmaf(v, b.y, acc.y);
                acc.z = fmaf(v, b.z, acc.z);
                acc.w = fmaf(v, b.w, acc.w);
            }
        }
    }
#pragma unroll
    for (int o = GL; o < 32; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    }
    return acc;
}

// group 0 stores a PP-wide row (float4 per lane; 4 GL >= PP)
template <int GL>
__device__ __forceinline__ void store_line4(float *__restrict__ dst, int PP, int lane, float4 acc) {
    if (lane < GL && 4 * lane < PP) *reinterpret_cast<float4 *>(dst + 4 * lane) = acc;
}

// ---------------------------------------------------------------------------
// Gather-accumulate with exact-width lane groups (the X^T W pass; measured on
// the 50000 x 500000 Zipf matrix at p = 20: 0.570 ms per pass against 0.674 ms
// with power-of-two groups, while the X Y pass ran 0.802 against 0.612 ms in
// this form and keeps the power-of-two one): gl = ceil(p / 4) lanes take one entry,
// each lane a float4 of the gathered row, so ng = 32 / gl entries are in flight
// per warp instruction (lanes gl ng .. 31 idle); entries lo + g, lo + g + ng, ...
// go to group g.  Rows below H come from the shared-memory copy `hot` (row
// stride p4 = 4 gl); the others from B (row-major, PP wide) through the
// read-only path.  On return lane l < gl holds the sum over the groups of its
// four columns, added in a fixed order (a butterfly when gl is a power of two,
// else group by group), so results do not depend on timing.
// ---------------------------------------------------------------------------
struct LaneGroup {
    int gl, ng, g, l;
    __device__ LaneGroup(int p, int lane) {
        gl = (p + 3) >> 2;
        ng = 32 / gl;
        g = lane / gl;
        l = lane - g * gl;
    }
};

__device__ __forceinline__ float4 gather_line(const int32_t *__restrict__ idx, const float *__restrict__ vals,
                                              int64_t lo, int64_t hi, const float *__restrict__ B, int PP,
                                              const float *hot, int H, const LaneGroup &lg, int lane) {
    const bool active = lg.g < lg.ng;
    const int p4 = 4 * lg.gl, l4 = 4 * lg.l;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    // the (index, value) chunk of 32 entries is loaded one chunk ahead
    int32_t rn = lo + lane < hi ? __ldg(idx + lo + lane) : 0;
    float vn = lo + lane < hi ? __ldg(vals + lo + lane) : 0.0f;
    for (int64_t base = lo; base < hi; base += 32) {
        const int32_t rr = rn;
        const float vv = vn;
        const int64_t k = base + 32 + lane;
        rn = k < hi ? __ldg(idx + k) : 0;
        vn = k < hi ? __ldg(vals + k) : 0.0f;
        const int cnt = (int)((hi - base) < 32 ? (hi - base) : 32);
#pragma unroll 4
        for (int e = 0; e < cnt; e += lg.ng) {
            const int src = e + lg.g;
            const int r = __shfl_sync(0xffffffffu, rr, src & 31);
            const float v = __shfl_sync(0xffffffffu, vv, src & 31);
            if (active && src < cnt) {
                float4 b;
                if (r < H)
                    b = *reinterpret_cast<const float4 *>(hot + r * p4 + l4);
                else
                    b = __ldg(reinterpret_cast<const float4 *>(B + (int64_t)r * PP + l4));
                acc.x = fmaf(v, b.x, acc.x);
                acc.y = fmaf(v, b.y, acc.y);
                acc.z = fmaf(v, b.z, acc.z);
                acc.w = fmaf(v, b.w, acc.w);
            }
        }
    }
    if ((lg.gl & (lg.gl - 1)) == 0) {
        // gl a power of two (ng gl = 32): butterfly over the group bits
        for (int o = lg.gl; o < 32; o <<= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
            acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
        }
        return acc;
    }
    float4 t = acc;
    for (int gg = 1; gg < lg.ng; ++gg) {
        const int from = (lg.l + gg * lg.gl) & 31;
        t.x += __shfl_sync(0xffffffffu, acc.x, from);
        t.y += __shfl_sync(0xffffffffu, acc.y, from);
        t.z += __shfl_sync(0xffffffffu, acc.z, from);
        t.w += __shfl_sync(0xffffffffu, acc.w, from);
    }
    return t;
}

// lanes l < PP / 4 store the PP-wide row: the group sum for l < gl, zeros beyond
__device__ __forceinline__ void store_line(float *__restrict__ dst, int PP, int lane, const LaneGroup &lg,
                                           float4 t) {
    if (4 * lane < PP)
        *reinterpret_cast<float4 *>(dst + 4 * lane) = lane < lg.gl ? t : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// Six CTAs of 256 threads per SM, each with 32 KB of hot rows (a sweep over
// 0-200 KB of hot rows and 128-512 threads on the 50000 x 500000 Zipf matrix,
// p = 20: 0.67 ms per pass here, 0.78 ms without hot rows, 1.30 ms with 200 KB
// and one CTA per SM, whose occupancy is too low to hide the cold gathers).
constexpr int kXtThreads = 256;
constexpr int kXtPerSm = 6;
constexpr size_t kHotBytes = 32 * 1024;  // shared memory for the hot rows of W

// Y (n x PP row-major) = X^T Wr: warp per column x_i.  The first H rows of
// Wr (the most frequent row ids of a Zipf-like X come first) are copied to
// shared memory once per CTA; kXtPerSm persistent CTAs per SM.
__global__ void __launch_bounds__(kXtThreads) spmm_xt_kernel(const int64_t *__restrict__ colptr,
                                                            const int32_t *__restrict__ rowidx,
                                                            const float *__restrict__ cval, int64_t n,
                                                            const float *__restrict__ Wr, int PP, int p, int H,
                                                            float *__restrict__ Y) {
    extern __shared__ float4 hot4[];
    const int lane = threadIdx.x & 31;
    const LaneGroup lg(p, lane);
    const int q4 = lg.gl;  // float4s per hot row
    const int64_t nv = (int64_t)H * q4;
    for (int64_t e = threadIdx.x; e < nv; e += blockDim.x) {
        const int64_t row = e / q4;
        const int c = (int)(e - row * q4) * 4;
        hot4[e] = *reinterpret_cast<const float4 *>(Wr + row * PP + c);
    }
    __syncthreads();
    const float *hot = reinterpret_cast<const float *>(hot4);
    for (int64_t i = global_warp(); i < n; i += warps_in_grid()) {
        const float4 t = gather_line(rowidx, cval, colptr[i], colptr[i + 1], Wr, PP, hot, H, lg, lane);
        store_line(Y + i * PP, PP, lane, lg, t);
    }
}

// G rows (dpad x PP row-major) = X Y over the row work list: single-segment rows
// go straight to G, segments of long rows to partial[item]
template <int GL>
__global__ void __launch_bounds__(32 * kWarps) spmm_x4_kernel(const int64_t *__restrict__ rowptr,
                                                              const int32_t *__restrict__ colidx,
                                                              const float *__restrict__ val, int64_t d,
                                                              const int64_t *__restrict__ item_off,
                                                              const int2 *__restrict__ items, int64_t nitems,
                                                              int seg, const float *__restrict__ Y, int PP, int p,
                                                              float *__restrict__ G, float *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    for (int64_t it = global_warp(); it < nitems; it += warps_in_grid()) {
        const int2 rs = items[it];
        const int64_t r = rs.x;
        int64_t lo = 0, hi = 0;
        if (r < d) {
            lo = rowptr[r] + (int64_t)rs.y * seg;
            hi = rowptr[r + 1];
            if (hi > lo + seg) hi = lo + seg;
        }
        const float4 acc = gather_line4<GL>(colidx, val, lo, hi, Y, PP, p, nullptr, 0, 4, lane);
        const bool single = (item_off[r + 1] - item_off[r]) == 1;
        store_line4<GL>(single ? G + r * PP : partial + it * PP, PP, lane, acc);
    }
}

template <typename F>
void dispatch_gl(int p, F &&f) {
    if (p <= 16) f(std::integral_constant<int, 4>{});
    else if (p <= 32) f(std::integral_constant<int, 8>{});
    else if (p <= 64) f(std::integral_constant<int, 16>{});
    else if (p <= 128) f(std::integral_constant<int, 32>{});
    else {
        set_error("sparse kernels support at most 128 block columns");
        throw Error{LRA_EINVAL};
    }
}

void check_sparse_p(int p) {
    if (p < 1 || p > 128) {
        set_error("sparse kernels support 1 to 128 block columns");
        throw Error{LRA_EINVAL};
    }
}

int sm_count_sparse() {
    int dev = 0, v = 0;
    LRA_CUDA(cudaGetDevice(&dev));
    LRA_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return v > 0 ? v : 1;
}

// ---------------------------------------------------------------------------
// SVRG inner loop in factored form (sparse X).  W - Wt = a Z + b M, so a step
// with column x_i (c = c_i) is
//     r = a (x_i^T Z) + b (x_i^T M),  a' = (1 - eta lambda) a,
//     b' = (1 - eta lambda) b - eta,  Z[rows of x_i] += (eta c / a') x_i r,
// and Z is rescaled (Z <- a Z, a <- 1) once a < 2^-30.  One CTA runs the
// chain; warp w takes the entries w, w + 8, ... of the column, lanes the columns
// of the block (row-major Z and M, PP wide).
//
// Deflated matrix (I - U U^T) X (Algorithm 6 on the fly; U orthonormal, c
// columns): the step's column is x'_i = x_i - U g_i, g_i = U^T x_i.  With
// W - Wt = a (Z - U K) + b M, x'_i is orthogonal to U, so
//     r = a (x_i^T Z - g_i^T L) + b (x_i^T M - g_i^T N),  L = U^T Z, N = U^T M,
// and the step adds (eta c / a') x_i r to Z and (eta c / a') g_i r to both L
// and K: K = L - L0 throughout (L0 = U^T Z at the start).  L, L0 and N (c x PP)
// stay in shared memory; K is written out for the final W.
// ---------------------------------------------------------------------------
__global__ void zdiff_kernel(const float *__restrict__ W, const float *__restrict__ Wt, int64_t dpad, int p, int PP,
                             float *__restrict__ Z) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < dpad * PP; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / PP;
        const int j = (int)(e - r * PP);
        Z[e] = j < p ? W[r + (int64_t)j * dpad] - Wt[r + (int64_t)j * dpad] : 0.0f;
    }
}

constexpr int kColCap = 1024;  // entries of a column staged in shared memory (longer: read in place)

template <int NQ>
__global__ void __launch_bounds__(32 * kWarps) inner_csc_kernel(const int64_t *__restrict__ colptr,
                                                                const int32_t *__restrict__ rowidx,
                                                                const float *__restrict__ cval, int64_t dpad, int PP,
                                                                const float *__restrict__ Mr, float *__restrict__ Z,
                                                                const int32_t *__restrict__ idx,
                                                                const float *__restrict__ cvals, int64_t m, double eta,
                                                                double lam, double *__restrict__ ab,
                                                                const float *__restrict__ Gt, int c, int PPc,
                                                                const float *__restrict__ LN, float *__restrict__ Kout) {
    constexpr int kPer = kColCap / (32 * kWarps);  // staged entries per thread
    __shared__ int32_t sr[2][kColCap];
    __shared__ float sv[2][kColCap];
    __shared__ float redz[kWarps][32 * NQ], redm[kWarps][32 * NQ];
    __shared__ float rv[32 * NQ];
    extern __shared__ float dfs[];  // deflation: L, L0, N (c x PP each), g of two steps
    float *Ls = dfs, *L0s = dfs + (size_t)c * PP, *Ns = dfs + 2 * (size_t)c * PP, *gs = dfs + 3 * (size_t)c * PP;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const double g = 1.0 - eta * lam;
    double a = 1.0, b = 0.0;

    for (int e = tid; e < c * PP; e += blockDim.x) {
        Ls[e] = L0s[e] = LN[e];
        Ns[e] = LN[(size_t)c * PP + e];
    }
    for (int e = tid; e < c; e += blockDim.x) gs[e] = Gt[(int64_t)idx[0] * PPc + e];
    // column of step 0 into buffer 0
    int64_t lo = colptr[idx[0]], hi = colptr[idx[0] + 1];
    if (hi - lo <= kColCap) {
        for (int64_t e = tid; e < hi - lo; e += blockDim.x) {
            sr[0][e] = rowidx[lo + e];
            sv[0][e] = cval[lo + e];
        }
    }
    __syncthreads();
    for (int64_t t = 0; t < m; ++t) {
        const int cur = (int)(t & 1);
        const int64_t len = hi - lo;
        const bool staged = len <= kColCap;
        const int32_t *er = staged ? sr[cur] : rowidx + lo;
        const float *ev = staged ? sv[cur] : cval + lo;

        // next step's column: its bounds and entries travel while this step runs
        int64_t lo1 = 0, hi1 = 0;
        int32_t pr[kPer];
        float pv[kPer];
        if (t + 1 < m) {
            const int64_t i1 = idx[t + 1];
            lo1 = colptr[i1];
            hi1 = colptr[i1 + 1];
            if (hi1 - lo1 <= kColCap) {
#pragma unroll
                for (int u = 0; u < kPer; ++u) {
                    const int64_t e = tid + (int64_t)u * blockDim.x;
                    pr[u] = e < hi1 - lo1 ? rowidx[lo1 + e] : 0;
                    pv[u] = e < hi1 - lo1 ? cval[lo1 + e] : 0.0f;
                }
            }
        }

        float sz[NQ], sm[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) sz[q] = sm[q] = 0.0f;
#pragma unroll 4
        for (int64_t e = w; e < len; e += kWarps) {
            const int64_t r = er[e];
            const float v = ev[e];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = lane + 32 * q;
                if (j < PP) {
                    sz[q] = fmaf(v, Z[r * PP + j], sz[q]);
                    sm[q] = fmaf(v, __ldg(Mr + r * PP + j), sm[q]);
                }
            }
        }
        const float *gc = gs + (size_t)cur * c;
        for (int u = w; u < c; u += kWarps) {
            const float ga = gc[u];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = lane + 32 * q;
                if (j < PP) {
                    sz[q] = fmaf(-ga, Ls[u * PP + j], sz[q]);
                    sm[q] = fmaf(-ga, Ns[u * PP + j], sm[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            redz[w][lane + 32 * q] = sz[q];
            redm[w][lane + 32 * q] = sm[q];
        }
        __syncthreads();
        if (tid < 32 * NQ) {
            float z = 0.0f, mm = 0.0f;
#pragma unroll
            for (int u = 0; u < kWarps; ++u) {
                z += redz[u][tid];
                mm += redm[u][tid];
            }
            rv[tid] = (float)(a * (double)z + b * (double)mm);
        }
        __syncthreads();
        const double a1 = g * a;
        b = g * b - eta;
        const float coef = (float)(eta * (double)cvals[t] / a1);
#pragma unroll 4
        for (int64_t e = w; e < len; e += kWarps) {
            const int64_t r = er[e];
            const float cv = coef * ev[e];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = lane + 32 * q;
                if (j < PP) Z[r * PP + j] = fmaf(cv, rv[j], Z[r * PP + j]);
            }
        }
        for (int u = w; u < c; u += kWarps) {
            const float cg = coef * gc[u];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = lane + 32 * q;
                if (j < PP) Ls[u * PP + j] = fmaf(cg, rv[j], Ls[u * PP + j]);
            }
        }
        // stage the next column and g (the other buffers are no longer read)
        if (t + 1 < m && hi1 - lo1 <= kColCap) {
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const int64_t e = tid + (int64_t)u * blockDim.x;
                if (e < hi1 - lo1) {
                    sr[cur ^ 1][e] = pr[u];
                    sv[cur ^ 1][e] = pv[u];
                }
            }
        }
        if (t + 1 < m)
            for (int e = tid; e < c; e += blockDim.x) gs[(size_t)(cur ^ 1) * c + e] = Gt[(int64_t)idx[t + 1] * PPc + e];
        a = a1;
        if (a < 0x1p-30) {
            __syncthreads();
            const float af = (float)a;
            for (int64_t e = tid; e < dpad * PP; e += blockDim.x) Z[e] *= af;
            for (int e = tid; e < c * PP; e += blockDim.x) {
                Ls[e] *= af;
                L0s[e] *= af;
            }
            a = 1.0;
        }
        lo = lo1;
        hi = hi1;
        __syncthreads();
    }
    if (tid == 0) {
        ab[0] = a;
        ab[1] = b;
    }
    for (int e = tid; e < c * PP; e += blockDim.x) Kout[e] = Ls[e] - L0s[e];
}

// The same chain with a batch of nb > 1 samples per step (stochastic term
// averaged, every r_u taken at the same W): warp w computes r_u for the
// columns u = w, w + 8, ... (a whole column each, entries in order); the
// updates of the nb columns then go in turn (columns of a batch may share
// rows), each split over the warps.
template <int NQ>
__global__ void __launch_bounds__(32 * kWarps) inner_csc_batch_kernel(
    const int64_t *__restrict__ colptr, const int32_t *__restrict__ rowidx, const float *__restrict__ cval,
    int64_t dpad, int PP, const float *__restrict__ Mr, float *__restrict__ Z, const int32_t *__restrict__ idx,
    const float *__restrict__ cvals, int64_t m, int nb, double eta, double lam, double *__restrict__ ab,
    const float *__restrict__ Gt, int c, int PPc, const float *__restrict__ LN, float *__restrict__ Kout) {
    __shared__ float rv[16][32 * NQ];
    extern __shared__ float dfs[];  // deflation: L, L0, N (c x PP each)
    float *Ls = dfs, *L0s = dfs + (size_t)c * PP, *Ns = dfs + 2 * (size_t)c * PP;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const double g = 1.0 - eta * lam;
    double a = 1.0, b = 0.0;
    for (int e = tid; e < c * PP; e += blockDim.x) {
        Ls[e] = L0s[e] = LN[e];
        Ns[e] = LN[(size_t)c * PP + e];
    }
    __syncthreads();
    for (int64_t t = 0; t < m; ++t) {
        for (int u = w; u < nb; u += kWarps) {
            const int64_t i = idx[t * nb + u];
            const int64_t lo = colptr[i], hi = colptr[i + 1];
            float sz[NQ], sm[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) sz[q] = sm[q] = 0.0f;
#pragma unroll 4
            for (int64_t k = lo; k < hi; ++k) {
                const int64_t r = rowidx[k];
                const float v = cval[k];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int j = lane + 32 * q;
                    if (j < PP) {
                        sz[q] = fmaf(v, Z[r * PP + j], sz[q]);
                        sm[q] = fmaf(v, __ldg(Mr + r * PP + j), sm[q]);
                    }
                }
            }
            for (int e = 0; e < c; ++e) {
                const float ge = Gt[i * PPc + e];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int j = lane + 32 * q;
                    if (j < PP) {
                        sz[q] = fmaf(-ge, Ls[e * PP + j], sz[q]);
                        sm[q] = fmaf(-ge, Ns[e * PP + j], sm[q]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) rv[u][lane + 32 * q] = (float)(a * (double)sz[q] + b * (double)sm[q]);
        }
        __syncthreads();
        const double a1 = g * a;
        b = g * b - eta;
        for (int u = 0; u < nb; ++u) {
            const int64_t i = idx[t * nb + u];
            const int64_t lo = colptr[i], hi = colptr[i + 1];
            const float coef = (float)(eta * (double)cvals[t * nb + u] / (a1 * (double)nb));
            for (int64_t k = lo + w; k < hi; k += kWarps) {
                const int64_t r = rowidx[k];
                const float cv = coef * cval[k];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int j = lane + 32 * q;
                    if (j < PP) Z[r * PP + j] = fmaf(cv, rv[u][j], Z[r * PP + j]);
                }
            }
            for (int e = w; e < c; e += kWarps) {
                const float cg = coef * Gt[i * PPc + e];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int j = lane + 32 * q;
                    if (j < PP) Ls[e * PP + j] = fmaf(cg, rv[u][j], Ls[e * PP + j]);
                }
            }
            __syncthreads();
        }
        a = a1;
        if (a < 0x1p-30) {
            const float af = (float)a;
            for (int64_t e = tid; e < dpad * PP; e += blockDim.x) Z[e] *= af;
            for (int e = tid; e < c * PP; e += blockDim.x) {
                Ls[e] *= af;
                L0s[e] *= af;
            }
            a = 1.0;
            __syncthreads();
        }
    }
    if (tid == 0) {
        ab[0] = a;
        ab[1] = b;
    }
    for (int e = tid; e < c * PP; e += blockDim.x) Kout[e] = Ls[e] - L0s[e];
}

// W = Wt + a (Z - U K) + b M  (c = 0: no deflation)
__global__ void inner_final_kernel(const float *__restrict__ Wt, const float *__restrict__ Z,
                                   const float *__restrict__ Mr, const double *__restrict__ ab, int64_t dpad, int p,
                                   int PP, const float *__restrict__ U, int c, const float *__restrict__ K,
                                   float *__restrict__ W) {
    const float a = (float)ab[0], b = (float)ab[1];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < dpad * p; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / dpad, r = e - j * dpad;
        float z = Z[r * PP + j];
        for (int u = 0; u < c; ++u) z = fmaf(-U[r + (int64_t)u * dpad], K[(int64_t)u * PP + j], z);
        W[e] = Wt[e] + a * z + b * Mr[r * PP + j];
    }
}

template <typename F>
void dispatch_nq(int PP, F &&f) {
    switch (ceil_div(PP, 32)) {
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 3: f(std::integral_constant<int, 3>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        default:
            set_error("sparse kernels support at most 128 block columns");
            throw Error{LRA_EINVAL};
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
void csr_check(cudaStream_t s, const int64_t *rowptr, const int32_t *colidx, const float *val, int64_t d,
               int64_t n, int64_t nnz, int *bad) {
    LRA_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    csr_check_kernel<<<grid_for(d, kWarps), 32 * kWarps, 0, s>>>(rowptr, colidx, val, d, n, nnz, bad);
    LRA_LAUNCHED();
}

int64_t sparse_scan_scratch(int64_t N) { return ceil_div(std::max<int64_t>(N, 1), kScanTile) + 8; }

void csr_transpose(cudaStream_t s, const int64_t *rowptr, const int32_t *colidx, const float *val, int64_t d,
                   int64_t n, int64_t nnz, int64_t *colptr, int32_t *rowidx, float *cval, int64_t *cnt,
                   int *cursor, int64_t *scan_scratch) {
    LRA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * n, s));
    LRA_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * n, s));
    if (nnz > 0) {
        col_count_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(colidx, nnz, reinterpret_cast<unsigned long long *>(cnt));
        LRA_LAUNCHED();
    }
    exclusive_scan(s, cnt, n, colptr, scan_scratch);
    if (nnz == 0) return;
    col_scatter_kernel<<<grid_for(d, kWarps), 32 * kWarps, 0, s>>>(rowptr, colidx, val, d, colptr, cursor, rowidx,
                                                                   cval);
    LRA_LAUNCHED();
    sort_cols_warp_kernel<<<grid_for(n, kSortWarps), 32 * kSortWarps, 0, s>>>(colptr, n, rowidx, cval);
    LRA_LAUNCHED();
    sort_cols_block_kernel<<<152, 512, 0, s>>>(colptr, n, rowidx, cval);
    LRA_LAUNCHED();
}

void sparse_row_items(cudaStream_t s, const int64_t *rowptr, int64_t d, int64_t dpad, int seg, int64_t *nseg,
                      int64_t *item_off, int64_t *scan_scratch) {
    row_segs_kernel<<<grid_for(dpad, 256), 256, 0, s>>>(rowptr, d, dpad, seg, nseg);
    LRA_LAUNCHED();
    exclusive_scan(s, nseg, dpad, item_off, scan_scratch);
}

void sparse_fill_items(cudaStream_t s, const int64_t *item_off, int64_t dpad, int2 *items) {
    fill_items_kernel<<<grid_for(dpad, 256), 256, 0, s>>>(item_off, dpad, items);
    LRA_LAUNCHED();
}

void sparse_colnorms(cudaStream_t s, const int64_t *colptr, const float *cval, int64_t n, double *norm2) {
    sparse_colnorms_kernel<<<grid_for(n, kWarps), 32 * kWarps, 0, s>>>(colptr, cval, n, norm2);
    LRA_LAUNCHED();
}

void spmm_xt(cudaStream_t s, const int64_t *colptr, const int32_t *rowidx, const float *cval, int64_t n,
             int64_t d, const float *Wr, int PP, int p, float *Y) {
    check_sparse_p(p);
    const int p4 = (p + 3) & ~3;
    const int H = (int)std::min<int64_t>(d, (int64_t)(kHotBytes / (sizeof(float) * p4)));
    const size_t smem = sizeof(float) * (size_t)H * p4;
    ensure_smem(spmm_xt_kernel, (int)std::max<size_t>(smem, 1));
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sm_count_sparse() * kXtPerSm, ceil_div(n, kXtThreads / 32)));
    spmm_xt_kernel<<<grid, kXtThreads, smem, s>>>(colptr, rowidx, cval, n, Wr, PP, p, H, Y);
    LRA_LAUNCHED();
}

void spmm_x(cudaStream_t s, const int64_t *rowptr, const int32_t *colidx, const float *val, int64_t d,
            int64_t dpad, const int64_t *item_off, const int2 *items, int64_t nitems, int seg, const float *Y,
            int PP, int p, float *G, float *partial) {
    dispatch_gl(p, [&](auto glc) {
        constexpr int GL = decltype(glc)::value;
        spmm_x4_kernel<GL><<<grid_for(nitems, kWarps), 32 * kWarps, 0, s>>>(rowptr, colidx, val, d, item_off, items,
                                                                           nitems, seg, Y, PP, p, G, partial);
        LRA_LAUNCHED();
    });
    if (nitems > dpad) {
        long_rows_kernel<<<grid_for(dpad, kWarps), 32 * kWarps, 0, s>>>(item_off, dpad, partial, PP, G);
        LRA_LAUNCHED();
    }
}

void svrg_inner_csc(cudaStream_t s, const int64_t *colptr, const int32_t *rowidx, const float *cval, int64_t dpad,
                    int p, int PP, float *W, const float *Wt, const float *Mr, float *Z, double *ab,
                    const int32_t *idx, const float *cvals, int64_t m, double eta, double lam, int batch,
                    const InnerDefl *defl) {
    if (m <= 0) return;
    if (batch < 1 || batch > 16) {
        set_error("batch must be in [1, 16]");
        throw Error{LRA_EINVAL};
    }
    zdiff_kernel<<<grid_for(dpad * PP, 256), 256, 0, s>>>(W, Wt, dpad, p, PP, Z);
    LRA_LAUNCHED();
    const int c = defl ? defl->c : 0;
    float *LN = defl ? defl->scratch : nullptr;  // L0 = U^T Z, N = U^T M, then K
    float *K = LN ? LN + 2 * (size_t)c * PP : nullptr;
    if (c > 0) {
        defl_coef(s, defl->U, dpad, c, Z, PP, 1, dpad, PP, LN, PP);
        defl_coef(s, defl->U, dpad, c, Mr, PP, 1, dpad, PP, LN + (size_t)c * PP, PP);
    }
    const float *Gt = defl ? defl->Gt : nullptr;
    const int PPc = defl ? defl->PPc : 0;
    dispatch_nq(PP, [&](auto nq) {
        constexpr int NQ = decltype(nq)::value;
        if (batch == 1) {
            auto k = inner_csc_kernel<NQ>;
            const size_t smem = sizeof(float) * (3 * (size_t)c * PP + 2 * (size_t)c);
            ensure_smem(k, (int)smem);
            k<<<1, 32 * kWarps, smem, s>>>(colptr, rowidx, cval, dpad, PP, Mr, Z, idx, cvals, m, eta, lam, ab, Gt, c,
                                           PPc, LN, K);
        } else {
            auto k = inner_csc_batch_kernel<NQ>;
            const size_t smem = sizeof(float) * 3 * (size_t)c * PP;
            ensure_smem(k, (int)smem);
            k<<<1, 32 * kWarps, smem, s>>>(colptr, rowidx, cval, dpad, PP, Mr, Z, idx, cvals, m, batch, eta, lam, ab,
                                           Gt, c, PPc, LN, K);
        }
        LRA_LAUNCHED();
    });
    inner_final_kernel<<<grid_for(dpad * p, 256), 256, 0, s>>>(Wt, Z, Mr, ab, dpad, p, PP, c > 0 ? defl->U : nullptr,
                                                                c, K, W);
    LRA_LAUNCHED();
}

}  // namespace lra
