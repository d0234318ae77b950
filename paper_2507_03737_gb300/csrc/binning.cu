// Tile binning and the (tile, depth) sort.
//
// The sort is a most-significant-digit radix sort whose first digit is the
// global tile id: the projection counts each tile's duplicates, an exclusive
// scan turns the counts into tile ranges (which are therefore final before any
// key moves), and the emission buckets every (depth bits << 32 | index) key
// into its tile's range through a per-tile cursor. The remaining digits are
// sorted inside each tile. Because every key within a tile is unique
// (depth bits, Gaussian index), the order inside a tile is fully determined
// even though the bucketing order is not: equal depths come out by ascending
// index, as a stable sort of the emission order would give. The scan uses three
// launches (block sums, scan of block sums, apply), so no block ever waits on
// another.
#include "s3gs_internal.cuh"

namespace s3gs {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned warp_incl_scan(unsigned x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block scan of one value per thread; returns the block total in *total.
__device__ __forceinline__ unsigned block_excl_scan(unsigned x, unsigned *s_warp, unsigned *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inc = warp_incl_scan(x);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
        unsigned wi = warp_incl_scan(w);
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    unsigned r = inc - x + s_warp[warp];
    *total = s_warp[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ unsigned load_count(const unsigned *c, long long i, long long n) {
    return i < n ? c[i] : 0u;
}

__global__ void __launch_bounds__(kScanThreads) scan_block_sums(const ScanArgs a) {
    __shared__ unsigned s_warp[33];
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += load_count(a.tile_count, base + k, a.n_tiles);
    unsigned tot;
    block_excl_scan(s, s_warp, &tot);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = tot;
}

// One block: exclusive scan of the block sums in 64-bit, total and overflow check.
__global__ void __launch_bounds__(kScanThreads) scan_partials(const ScanArgs a, int n_parts) {
    __shared__ unsigned long long s_carry;
    __shared__ unsigned s_warp[33];
    if (threadIdx.x == 0) s_carry = 0ull;
    __syncthreads();
    for (int base = 0; base < n_parts; base += kScanThreads) {
        int i = base + threadIdx.x;
        unsigned x = i < n_parts ? a.partials[i] : 0u;
        unsigned tot;
        unsigned ex = block_excl_scan(x, s_warp, &tot);
        unsigned long long c = s_carry;
        unsigned long long off = c + ex;
        // a tile offset must fit in 32 bits; larger totals are reported as overflow
        if (i < n_parts) a.partials[i] = off > 0xffffffffull ? 0xffffffffu : (unsigned)off;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = c + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        unsigned long long K = s_carry;
        a.ctr->n_dup = K;
        a.ctr->overflow = (K > a.key_capacity || K > (unsigned long long)S3GS_MAX_DUPLICATES) ? 1u : 0u;
        a.tile_start[a.n_tiles] = K > 0xffffffffull ? 0xffffffffu : (unsigned)K;  // end sentinel
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply(const ScanArgs a) {
    __shared__ unsigned s_warp[33];
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    unsigned v[kScanItems];
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = load_count(a.tile_count, base + k, a.n_tiles);
        s += v[k];
    }
    unsigned tot;
    unsigned ex = block_excl_scan(s, s_warp, &tot) + a.partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + k;
        if (i < a.n_tiles) {
            a.tile_start[i] = ex;
            a.cursor[i] = ex;
        }
        ex += v[k];
    }
}

// One warp expands the (record, tile) pairs of its 32 records: an inclusive
// warp scan of the records' tile counts numbers the pairs, and each round every
// lane takes one pair (found by a 5-step search of the scan), so all lanes stay
// busy whatever the mix of visible, culled, small and large records. Four rounds
// of cursor atomics are issued before their results are consumed.
__global__ void __launch_bounds__(256) emit_kernel(const EmitArgs a, const __grid_constant__ ViewBatch vb) {
    __shared__ unsigned s_incl[8][32], s_excl[8][32], s_origin[8][32], s_ntx[8][32], s_tx[8][32];
    __shared__ unsigned long long s_key[8][32];
    if (a.ctr->overflow) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)vb.n_views * a.n;
    unsigned cnt = 0, origin = 0, ntx = 1, tiles_x = 0;
    unsigned long long key = 0;
    if (r < total) {
        const int2 ext = a.ext[r];
        if (ext.x > 0) {
            const int v = (int)(r / a.n);
            const unsigned g = (unsigned)(r - (long long)v * a.n);
            const ViewInfo &vi = vb.v[v];
            const float4 ra = a.rec[r].a;
            const float z = a.rec[r].b.z;
            const float x0 = ceilf(__fsub_rn(ra.x, (float)ext.x)), x1 = floorf(__fadd_rn(ra.x, (float)ext.x));
            const float y0 = ceilf(__fsub_rn(ra.y, (float)ext.y)), y1 = floorf(__fadd_rn(ra.y, (float)ext.y));
            const int tx0 = (x0 > 0.f ? (int)x0 : 0) / vb.tile_w;
            const int tx1 = (x1 < (float)(vi.w - 1) ? (int)x1 : vi.w - 1) / vb.tile_w;
            const int ty0 = (y0 > 0.f ? (int)y0 : 0) / vb.tile_h;
            const int ty1 = (y1 < (float)(vi.h - 1) ? (int)y1 : vi.h - 1) / vb.tile_h;
            ntx = (unsigned)(tx1 - tx0 + 1);
            cnt = ntx * (unsigned)(ty1 - ty0 + 1);
            origin = (unsigned)(vi.tile_base + ty0 * vi.tiles_x + tx0);
            tiles_x = (unsigned)vi.tiles_x;
            key = ((unsigned long long)__float_as_uint(z) << 32) | g;
        }
    }
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned wtotal = __shfl_sync(0xffffffffu, incl, 31);
    if (wtotal == 0) return;
    s_incl[warp][lane] = incl;
    s_excl[warp][lane] = incl - cnt;
    s_origin[warp][lane] = origin;
    s_ntx[warp][lane] = ntx;
    s_tx[warp][lane] = tiles_x;
    s_key[warp][lane] = key;
    __syncwarp();
    for (unsigned base = 0; base < wtotal; base += 4 * 32) {
        unsigned pos[4];
        unsigned long long kk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned j = base + u * 32 + lane;
            pos[u] = 0xffffffffu;
            if (j < wtotal) {
                unsigned src = 0;
#pragma unroll
                for (unsigned b = 16; b > 0; b >>= 1)
                    if (s_incl[warp][src + b - 1] <= j) src += b;
                const unsigned local = j - s_excl[warp][src];
                const unsigned nx = s_ntx[warp][src];
                const unsigned tile = s_origin[warp][src] + (local / nx) * s_tx[warp][src] + (local % nx);
                pos[u] = atomicAdd(a.cursor + tile, 1u);
                kk[u] = s_key[warp][src];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (pos[u] < a.key_capacity) a.keys[pos[u]] = kk[u];
    }
}

// ---- per-tile sort ----
// Bitonic network in the "all comparators ascending" form: for each block size
// s the first step compares element i with its mirror in the block, the
// following steps compare i with i + d for d = s/4 ... 1. Every comparator puts
// the smaller key at the lower index, so virtual +inf padding past the end of a
// segment never moves and comparators that reach past the end are skipped.
constexpr int kSortThreads = 512;
constexpr int kSortCap = 4096;  // keys sorted entirely in shared memory (32 KB)

__device__ __forceinline__ void cswap(unsigned long long *k, unsigned i, unsigned j) {
    unsigned long long x = k[i], y = k[j];
    if (x > y) {
        k[i] = y;
        k[j] = x;
    }
}

// Full network over a segment of length n <= cap held at `k` (shared or global).
__device__ void bitonic_full(unsigned long long *k, unsigned n) {
    for (unsigned s = 2; s < 2 * n; s <<= 1) {
        unsigned half = s >> 1;
        for (unsigned t = threadIdx.x; t < ((n + 1) >> 1) + half; t += blockDim.x) {
            unsigned blk = t / half, off = t % half;
            unsigned i = blk * s + off, j = blk * s + s - 1 - off;
            if (j < n) cswap(k, i, j);
        }
        __syncthreads();
        for (unsigned d = half >> 1; d > 0; d >>= 1) {
            for (unsigned t = threadIdx.x; t < ((n + 1) >> 1) + d; t += blockDim.x) {
                unsigned blk = t / d, off = t % d;
                unsigned i = blk * 2 * d + off, j = i + d;
                if (j < n) cswap(k, i, j);
            }
            __syncthreads();
        }
    }
}

// Half-cleaner steps d = d0, d0/2, ..., 1 within a segment of length n.
__device__ void bitonic_cleaners(unsigned long long *k, unsigned n, unsigned d0) {
    for (unsigned d = d0; d > 0; d >>= 1) {
        for (unsigned t = threadIdx.x; t < ((n + 1) >> 1) + d; t += blockDim.x) {
            unsigned blk = t / d, off = t % d;
            unsigned i = blk * 2 * d + off, j = i + d;
            if (j < n) cswap(k, i, j);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSortThreads) tile_sort_kernel(const SortArgs a) {
    __shared__ unsigned long long s_k[kSortCap];
    if (a.ctr->overflow) return;
    long long t = blockIdx.x;
    unsigned start = a.tile_start[t], end = a.tile_start[t + 1];
    unsigned n = end - start;
    if (n <= 1) return;
    unsigned long long *g = a.keys + start;
    if (n <= (unsigned)kSortCap) {
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) s_k[i] = g[i];
        __syncthreads();
        bitonic_full(s_k, n);
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) g[i] = s_k[i];
        return;
    }
    // Heavy tile: the first log2(cap) stages of the network stay inside aligned
    // chunks of `cap` keys and run in shared memory; every later stage runs its
    // long-distance steps in global memory and finishes each chunk in shared.
    for (unsigned c0 = 0; c0 < n; c0 += kSortCap) {
        unsigned m = min((unsigned)kSortCap, n - c0);
        for (unsigned i = threadIdx.x; i < m; i += blockDim.x) s_k[i] = g[c0 + i];
        __syncthreads();
        bitonic_full(s_k, m);
        for (unsigned i = threadIdx.x; i < m; i += blockDim.x) g[c0 + i] = s_k[i];
        __syncthreads();
    }
    for (unsigned s = 2 * kSortCap; s < 2 * n; s <<= 1) {
        unsigned half = s >> 1;
        for (unsigned tt = threadIdx.x; tt < ((n + 1) >> 1) + half; tt += blockDim.x) {
            unsigned blk = tt / half, off = tt % half;
            unsigned i = blk * s + off, j = blk * s + s - 1 - off;
            if (j < n) cswap(g, i, j);
        }
        __syncthreads();
        for (unsigned d = half >> 1; d >= (unsigned)kSortCap; d >>= 1) {
            for (unsigned tt = threadIdx.x; tt < ((n + 1) >> 1) + d; tt += blockDim.x) {
                unsigned blk = tt / d, off = tt % d;
                unsigned i = blk * 2 * d + off, j = i + d;
                if (j < n) cswap(g, i, j);
            }
            __syncthreads();
        }
        for (unsigned c0 = 0; c0 < n; c0 += kSortCap) {
            unsigned m = min((unsigned)kSortCap, n - c0);
            for (unsigned i = threadIdx.x; i < m; i += blockDim.x) s_k[i] = g[c0 + i];
            __syncthreads();
            bitonic_cleaners(s_k, m, kSortCap / 2);
            for (unsigned i = threadIdx.x; i < m; i += blockDim.x) g[c0 + i] = s_k[i];
            __syncthreads();
        }
    }
}

// ---- heaviest-first tile order for the persistent blend grid ----
__device__ __forceinline__ int load_bucket(unsigned cnt) { return cnt ? 32 - __clz(cnt) : 0; }  // 0..32

__global__ void tile_bucket_count(const OrderArgs a) {
    __shared__ unsigned s_c[33];
    for (int i = threadIdx.x; i < 33; i += blockDim.x) s_c[i] = 0;
    __syncthreads();
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_tiles;
         t += (long long)gridDim.x * blockDim.x)
        atomicAdd(&s_c[load_bucket(a.tile_start[t + 1] - a.tile_start[t])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < 33; i += blockDim.x)
        if (s_c[i]) atomicAdd(&a.bucket_cnt[i], s_c[i]);
}

__global__ void tile_bucket_scan(const OrderArgs a) {
    // heaviest bucket first: cursor[b] = sum of counts of buckets > b
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = 32; b >= 0; --b) {
            unsigned c = a.bucket_cnt[b];
            a.bucket_cnt[b] = acc;
            acc += c;
        }
    }
}

__global__ void tile_bucket_scatter(const OrderArgs a) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_tiles;
         t += (long long)gridDim.x * blockDim.x) {
        int b = load_bucket(a.tile_start[t + 1] - a.tile_start[t]);
        unsigned pos = atomicAdd(&a.bucket_cnt[b], 1u);
        a.order[pos] = (unsigned)t;
    }
}

}  // namespace

cudaError_t launch_scan(const ScanArgs &a, cudaStream_t s) {
    int n_parts = (int)((a.n_tiles + kScanTile - 1) / kScanTile);
    if (n_parts < 1) n_parts = 1;
    scan_block_sums<<<n_parts, kScanThreads, 0, s>>>(a);
    scan_partials<<<1, kScanThreads, 0, s>>>(a, n_parts);
    scan_apply<<<n_parts, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_emit(const EmitArgs &a, const ViewBatch &vb, cudaStream_t s) {
    long long total = (long long)vb.n_views * a.n;
    if (total == 0) return cudaSuccess;
    emit_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a, vb);
    return cudaGetLastError();
}

cudaError_t launch_tile_sort(const SortArgs &a, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    tile_sort_kernel<<<(unsigned)a.n_tiles, kSortThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const OrderArgs &a, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.bucket_cnt, 0, 33 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    int grid = (int)min((a.n_tiles + 255) / 256, 1024LL);
    if (grid < 1) grid = 1;
    tile_bucket_count<<<grid, 256, 0, s>>>(a);
    tile_bucket_scan<<<1, 32, 0, s>>>(a);
    tile_bucket_scatter<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace s3gs
