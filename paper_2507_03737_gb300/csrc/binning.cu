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

// One warp expands the (record, tile) pairs of its 32 records in the two levels
// of the projection's count: level 1 numbers the tile rows of the records'
// bounding rectangles (a warp scan) and every lane computes one row's span of
// covered tile columns with the same row_span the count used; level 2 numbers
// the round's covered tiles and every lane emits one key per sub-round. All lanes
// stay busy whatever the mix of visible, culled, small and large records, and
// only covered tiles cost a cursor atomic. Four sub-rounds of cursor atomics
// are issued before their results are consumed. A round whose rows are all short
// (at most kRowSeqMax tiles, the common case for small Gaussians) skips level 2:
// each lane expands its own row, four tiles at a time.
//
// With the occlusion cut the same enumeration first runs in COUNT mode (after the
// cut, before the scan), counting only the pairs in front of their tile's cut. A
// record behind its view's largest cut is skipped whole, a row behind the row's
// largest cut costs no level-2 work, and each pair is checked against its tile's cut.
constexpr unsigned kRowSeqMax = 16;  // longest tile row a lane expands by itself (a round of longer rows is spread over the warp)

template <bool COUNT>
__global__ void __launch_bounds__(256) emit_kernel(const EmitArgs a, const __grid_constant__ ViewBatch vb) {
    __shared__ unsigned s_incl[8][32], s_excl[8][32], s_t0[8][32], s_ntx[8][32], s_orig[8][32];
    __shared__ unsigned long long s_key[8][32];
    __shared__ CoverEllipse s_ell[8][32];  // cover ellipse of the source record
    if (!COUNT && a.ctr->overflow) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // blockIdx.y is the view, so no record index needs dividing
    const int v = (int)blockIdx.y;
    const ViewInfo &vi = vb.v[v];
    const long long gl = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long r = (long long)v * a.n + gl;
    unsigned nrows = 0, ntx = 1, t0 = 0, orig = 0;
    unsigned long long key = 0;
    CoverEllipse ell;
    ell.u = ell.v = ell.B = ell.iA = ell.Aqc = ell.det = ell.yL = ell.mq = 0.f;
    ell.ym = -1.0f;
    if (gl < a.n) {
        const int2 ext = a.ext[r];
        const float4 rb = ext.x > 0 ? a.rec[r].b : make_float4(0.f, 0.f, 0.f, 0.f);
        // a record behind every cut of its view lists nowhere
        if (ext.x > 0 && !(a.cut && (unsigned)depth_bin(rb.z) > a.view_max[v])) {
            const unsigned g = (unsigned)gl;
            const float4 ra = a.rec[r].a;
            const float z = rb.z;
            ell = cover_ellipse(ra.x, ra.y, ra.z, ra.w, rb.x, a.rec[r].c.w);
            const float x0 = ceilf(__fsub_rn(ra.x, (float)ext.x)), x1 = floorf(__fadd_rn(ra.x, (float)ext.x));
            const float y0 = ceilf(__fsub_rn(ra.y, (float)ext.y)), y1 = floorf(__fadd_rn(ra.y, (float)ext.y));
            const int tx0 = tile_of(x0 > 0.f ? (int)x0 : 0, vb.tile_w);
            const int tx1 = tile_of(x1 < (float)(vi.w - 1) ? (int)x1 : vi.w - 1, vb.tile_w);
            const int ty0 = tile_of(y0 > 0.f ? (int)y0 : 0, vb.tile_h);
            const int ty1 = tile_of(y1 < (float)(vi.h - 1) ? (int)y1 : vi.h - 1, vb.tile_h);
            ntx = (unsigned)(tx1 - tx0 + 1);
            nrows = (unsigned)(ty1 - ty0 + 1);
            t0 = (unsigned)tx0 | ((unsigned)ty0 << 16);
            orig = (unsigned)(vi.tile_base + ty0 * vi.tiles_x) * kDepthBins + (unsigned)depth_bin(z);
            key = ((unsigned long long)__float_as_uint(z) << 32) | g;
        }
    }
    const unsigned incl = warp_incl_scan(nrows);
    const unsigned wtotal = __shfl_sync(0xffffffffu, incl, 31);
    if (wtotal == 0) return;
    s_incl[warp][lane] = incl;
    s_excl[warp][lane] = incl - nrows;
    s_t0[warp][lane] = t0;
    s_ntx[warp][lane] = ntx;
    s_orig[warp][lane] = orig;
    s_key[warp][lane] = key;
    s_ell[warp][lane] = ell;
    __syncwarp();
    const float inv_tw = __frcp_rn((float)vb.tile_w);  // exact: the tile width is a power of two
    const unsigned row_stride = (unsigned)vi.tiles_x * kDepthBins;
    for (unsigned base = 0; base < wtotal; base += 32) {
        const unsigned j = base + lane;
        int c0 = 0;
        unsigned len = 0, rowbase = 0;
        unsigned long long rkey = 0;
        if (j < wtotal) {
            unsigned src = 0;
#pragma unroll
            for (unsigned b = 16; b > 0; b >>= 1)
                if (s_incl[warp][src + b - 1] <= j) src += b;
            const unsigned row = j - s_excl[warp][src];
            rowbase = s_orig[warp][src] + row * row_stride;
            // the row's largest cut sits at its first tile
            if (!a.cut || (rowbase & (kDepthBins - 1)) <= a.row_max[rowbase / kDepthBins]) {
                const unsigned tt = s_t0[warp][src];
                const int ty = (int)(tt >> 16) + (int)row;
                const int py0 = ty * vb.tile_h, py1 = min(py0 + vb.tile_h - 1, vi.h - 1);
                const int cx0 = (int)(tt & 0xffffu);
                const int2 span = row_span(s_ell[warp][src], py0, py1, cx0, cx0 + (int)s_ntx[warp][src] - 1, inv_tw);
                c0 = span.x;
                len = span.y >= span.x ? (unsigned)(span.y - span.x + 1) : 0u;
                rkey = s_key[warp][src];
            }
        }
        const unsigned maxlen = __reduce_max_sync(0xffffffffu, len);
        if (maxlen <= kRowSeqMax) {
            // short rows: each lane takes its own row's tiles, four
            // at a time, rather than spreading the round's tiles over the warp
            for (unsigned q0 = 0; q0 < maxlen; q0 += 4) {
                unsigned pos[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned q = q0 + (unsigned)u;
                    const unsigned bucket = rowbase + (unsigned)(c0 + (int)q) * kDepthBins;
                    pos[u] = 0xffffffffu;
                    if (q < len && (!a.cut || (bucket & (kDepthBins - 1)) <= a.cut[bucket / kDepthBins])) {
                        if (COUNT) atomicAdd(a.tile_count + bucket, 1u);
                        else pos[u] = atomicAdd(a.cursor + bucket, 1u);
                    }
                }
                if (!COUNT) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (pos[u] < a.key_capacity) a.keys[pos[u]] = rkey;
                }
            }
            continue;
        }
        const unsigned incl2 = warp_incl_scan(len);
        const unsigned tot2 = __shfl_sync(0xffffffffu, incl2, 31);
        const unsigned excl2 = incl2 - len;
        if (COUNT) {
            for (unsigned b2 = 0; b2 < tot2; b2 += 32) {
                const unsigned j2 = b2 + lane;
                const int src2 = warp_find(incl2, j2);
                const int h0 = __shfl_sync(0xffffffffu, c0, src2);
                const unsigned he = __shfl_sync(0xffffffffu, excl2, src2);
                const unsigned hb = __shfl_sync(0xffffffffu, rowbase, src2);
                const unsigned bucket = hb + (unsigned)(h0 + (int)(j2 - he)) * kDepthBins;
                if (j2 < tot2 && (bucket & (kDepthBins - 1)) <= a.cut[bucket / kDepthBins])
                    atomicAdd(a.tile_count + bucket, 1u);
            }
            continue;
        }
        for (unsigned b2 = 0; b2 < tot2; b2 += 4 * 32) {
            unsigned pos[4];
            unsigned long long kk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned j2 = b2 + u * 32 + lane;
                const int src2 = warp_find(incl2, j2);
                const int h0 = __shfl_sync(0xffffffffu, c0, src2);
                const unsigned he = __shfl_sync(0xffffffffu, excl2, src2);
                const unsigned hb = __shfl_sync(0xffffffffu, rowbase, src2);
                kk[u] = __shfl_sync(0xffffffffu, rkey, src2);
                pos[u] = 0xffffffffu;
                const unsigned bucket = hb + (unsigned)(h0 + (int)(j2 - he)) * kDepthBins;
                // behind its tile's occlusion cut a pair is not listed
                if (j2 < tot2 && (!a.cut || (bucket & (kDepthBins - 1)) <= a.cut[bucket / kDepthBins]))
                    pos[u] = atomicAdd(a.cursor + bucket, 1u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (pos[u] < a.key_capacity) a.keys[pos[u]] = kk[u];
        }
    }
}

// ---- occlusion cut ----
// One warp per tile: lane l holds depth bins 8l..8l+7 of the tile's optical-depth
// sums; a warp scan finds the first bin at which the running sum reaches the
// threshold, which is the last bin the tile lists. Its largest value over each tile
// row is kept at the row's first tile (row_max) and over each view (view_max), both
// zeroed before, so the count and the emission can pass over whole rows and records
// that lie behind every cut they could meet.
__global__ void __launch_bounds__(256) cut_kernel(const CutArgs a, const __grid_constant__ ViewBatch vb) {
    const long long t = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= a.n_tiles) return;
    const int lane = threadIdx.x & 31;
    const uint4 *src = reinterpret_cast<const uint4 *>(a.occl + t * kDepthBins + lane * 8);
    const uint4 w0 = src[0], w1 = src[1];
    const unsigned o[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    unsigned long long run[8];
    unsigned long long acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) run[k] = (acc += o[k]);
    unsigned long long incl = acc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const unsigned long long excl = incl - acc;
    int first = kDepthBins - 1;
#pragma unroll
    for (int k = 7; k >= 0; --k)
        if (excl + run[k] >= kOcclThreshold) first = lane * 8 + k;
    const unsigned b = __reduce_min_sync(0xffffffffu, (unsigned)first);
    if (lane == 0) {
        a.cut[t] = (unsigned char)b;
        int v = 0;
        while (v + 1 < vb.n_views && vb.v[v + 1].tile_base <= t) ++v;
        const ViewInfo &vi = vb.v[v];
        const int ty = (int)(t - vi.tile_base) / vi.tiles_x;
        atomicMax(a.row_max + vi.tile_base + ty * vi.tiles_x, b);
        atomicMax(a.view_max + v, b);
    }
}

// ---- per-tile sort ----
// Bitonic network in the "all comparators ascending" form: for each block size
// s the first step compares element i with its mirror in the block, the
// following steps compare i with i + d for d = s/4 ... 1. Every comparator puts
// the smaller key at the lower index, so virtual +inf padding past the end of a
// segment never moves and comparators that reach past the end can be skipped.
// Steps whose partner lies in the same aligned 64-key block run in registers:
// a warp holds such a block as two keys per lane and exchanges them with warp
// shuffles; only the longer steps go through shared memory with block barriers.
constexpr int kSortThreads = 256;
constexpr int kSortCap = 4096;  // keys sorted entirely in shared memory (32 KB)
constexpr unsigned kSegKeys = 24;  // window that merges buckets into segments for the warp sorts
constexpr unsigned long long kInfKey = ~0ull;

__device__ __forceinline__ unsigned ceil_log2(unsigned n) { return n <= 1 ? 0 : 32 - __clz(n - 1); }

__device__ __forceinline__ void cswap(unsigned long long *k, unsigned i, unsigned j) {
    unsigned long long x = k[i], y = k[j];
    if (x > y) {
        k[i] = y;
        k[j] = x;
    }
}

__device__ __forceinline__ void cas_local(unsigned long long &lo, unsigned long long &hi) {
    const unsigned long long a = lo < hi ? lo : hi, b = lo < hi ? hi : lo;
    lo = a;
    hi = b;
}

// One comparator step on a register-held 64-key block (x0, x1) = keys
// (2 lane, 2 lane + 1). flip: partner = e ^ (2m + 1); otherwise partner = e ^ 2m
// (or e ^ 1 when m = 0).
__device__ __forceinline__ void reg_step(unsigned long long &x0, unsigned long long &x1, unsigned m, bool flip) {
    const unsigned lane = threadIdx.x & 31u;
    if (m == 0) {
        cas_local(x0, x1);
        return;
    }
    const unsigned long long y0 = __shfl_xor_sync(0xffffffffu, flip ? x1 : x0, m);
    const unsigned long long y1 = __shfl_xor_sync(0xffffffffu, flip ? x0 : x1, m);
    const unsigned top = flip ? (m + 1) >> 1 : m;  // highest bit in which the two lanes differ
    const bool lower = (lane & top) == 0;
    x0 = lower ? (x0 < y0 ? x0 : y0) : (x0 < y0 ? y0 : x0);
    x1 = lower ? (x1 < y1 ? x1 : y1) : (x1 < y1 ? y1 : x1);
}

// Stages s = 2 .. min(64, N) of a register-held block.
__device__ __forceinline__ void reg_stages(unsigned long long &x0, unsigned long long &x1, unsigned lsmax) {
    for (unsigned ls = 1; ls <= lsmax; ++ls) {
        reg_step(x0, x1, ((1u << ls) - 1) >> 1, true);
        for (int ld = (int)ls - 2; ld >= 0; --ld) reg_step(x0, x1, (1u << ld) >> 1, false);
    }
}

// Cleaner steps d = 32 .. 1 of a register-held block.
__device__ __forceinline__ void reg_cleaners(unsigned long long &x0, unsigned long long &x1) {
    for (int ld = 5; ld >= 0; --ld) reg_step(x0, x1, (1u << ld) >> 1, false);
}

__device__ void sort_pow2_smem(unsigned long long *k, unsigned lgN) {
    const unsigned N = 1u << lgN, lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned nblk = N >> 6;
    const unsigned first = lgN < 6 ? lgN : 6;
    for (unsigned b = warp; b < (nblk > 0 ? nblk : 1); b += nw) {
        unsigned long long x0 = k[(b << 6) + 2 * lane], x1 = k[(b << 6) + 2 * lane + 1];
        reg_stages(x0, x1, first);
        k[(b << 6) + 2 * lane] = x0;
        k[(b << 6) + 2 * lane + 1] = x1;
    }
    __syncthreads();
    for (unsigned ls = 7; ls <= lgN; ++ls) {
        const unsigned lh = ls - 1, half = 1u << lh;
        for (unsigned t = threadIdx.x; t < (N >> 1); t += blockDim.x) {
            const unsigned blk = t >> lh, off = t & (half - 1);
            cswap(k, (blk << ls) + off, (blk << ls) + (1u << ls) - 1 - off);
        }
        __syncthreads();
        for (int ld = (int)ls - 2; ld >= 6; --ld) {
            const unsigned d = 1u << ld;
            for (unsigned t = threadIdx.x; t < (N >> 1); t += blockDim.x) {
                const unsigned i = ((t >> ld) << (ld + 1)) + (t & (d - 1));
                cswap(k, i, i + d);
            }
            __syncthreads();
        }
        for (unsigned b = warp; b < nblk; b += nw) {
            unsigned long long x0 = k[(b << 6) + 2 * lane], x1 = k[(b << 6) + 2 * lane + 1];
            reg_cleaners(x0, x1);
            k[(b << 6) + 2 * lane] = x0;
            k[(b << 6) + 2 * lane + 1] = x1;
        }
        __syncthreads();
    }
}


// ---- register sort of up to 32 R keys by one warp (R keys per lane) ----
// Key e = R lane + h. A comparator whose partner differs from e only in the low
// log2(R) bits runs inside the lane; otherwise the partner lane is found with a
// shuffle (flip steps also mirror h).
__device__ __forceinline__ unsigned long long pick(bool lower, unsigned long long a, unsigned long long b) {
    const bool gt = a > b;
    return (gt == lower) ? b : a;  // lower: min(a, b); upper: max(a, b)
}

template <int R, int M>
__device__ __forceinline__ void inlane_step(unsigned long long (&x)[R]) {
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const int hp = h ^ M;
        if (hp > h) cas_local(x[h], x[hp]);
    }
}

// One comparator step of the network: partner = e ^ M (a flip step, which also
// mirrors h) or e ^ M for a power of two M (a cleaner step). M is known at
// compile time, so a whole network unrolls into straight-line shuffles and
// selects.
template <int R, unsigned M, bool FLIP>
__device__ __forceinline__ void regR_step(unsigned long long (&x)[R]) {
    if constexpr (M < (unsigned)R) {
        inlane_step<R, (int)M>(x);
    } else {
        const unsigned lane = threadIdx.x & 31u;
        unsigned long long y[R];
        if constexpr (FLIP) {
            constexpr unsigned lm = (M + 1) / R - 1, top = ((M + 1) / R) >> 1;
            const bool lower = (lane & top) == 0;
#pragma unroll
            for (int h = 0; h < R; ++h) y[h] = __shfl_xor_sync(0xffffffffu, x[h ^ (R - 1)], lm);
#pragma unroll
            for (int h = 0; h < R; ++h) x[h] = pick(lower, x[h], y[h]);
        } else {
            constexpr unsigned lm = M / R;
            const bool lower = (lane & lm) == 0;
#pragma unroll
            for (int h = 0; h < R; ++h) y[h] = __shfl_xor_sync(0xffffffffu, x[h], lm);
#pragma unroll
            for (int h = 0; h < R; ++h) x[h] = pick(lower, x[h], y[h]);
        }
    }
}

template <int R, int LD>
__device__ __forceinline__ void net_cleaners(unsigned long long (&x)[R]) {
    if constexpr (LD >= 0) {
        regR_step<R, (1u << LD), false>(x);
        net_cleaners<R, LD - 1>(x);
    }
}

template <int R, int LS, int LSMAX>
__device__ __forceinline__ void net_stages(unsigned long long (&x)[R]) {
    if constexpr (LS <= LSMAX) {
        regR_step<R, (1u << LS) - 1, true>(x);
        net_cleaners<R, LS - 2>(x);
        net_stages<R, LS + 1, LSMAX>(x);
    }
}

// Sort of one key segment of length n <= 2^LSMAX <= 32 R by one warp with an
// unrolled network.
template <int R, int LSMAX>
__device__ __forceinline__ void sort_segment_net(unsigned long long *g, unsigned n) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long x[R];
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const unsigned e = R * lane + h;
        x[h] = e < n ? g[e] : kInfKey;
    }
    net_stages<R, 1, LSMAX>(x);
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const unsigned e = R * lane + h;
        if (e < n) g[e] = x[h];
    }
}

// Warp sort of a segment of 2 <= n <= 128 keys: the network of the smallest
// power of two that holds it, one key per lane up to 32 keys.
__device__ __forceinline__ void sort_segment_warp(unsigned long long *g, unsigned n) {
    switch (ceil_log2(n)) {
    case 1: sort_segment_net<1, 1>(g, n); break;
    case 2: sort_segment_net<1, 2>(g, n); break;
    case 3: sort_segment_net<1, 3>(g, n); break;
    case 4: sort_segment_net<1, 4>(g, n); break;
    case 5: sort_segment_net<1, 5>(g, n); break;
    case 6: sort_segment_net<2, 6>(g, n); break;
    default: sort_segment_net<4, 7>(g, n); break;
    }
}

// Sort of one key segment of length n > 64 by the whole block (call uniformly).
__device__ void sort_segment_block(unsigned long long *g, unsigned n, unsigned long long *s_k) {
    const unsigned lane = threadIdx.x & 31u;
    if (n <= (unsigned)kSortCap) {
        const unsigned lgN = ceil_log2(n), N = 1u << lgN;
        for (unsigned i = threadIdx.x; i < N; i += blockDim.x) s_k[i] = i < n ? g[i] : kInfKey;
        __syncthreads();
        sort_pow2_smem(s_k, lgN);
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) g[i] = s_k[i];
        __syncthreads();
        return;
    }
    // Heavy segment: chunks of kSortCap keys are sorted in shared memory (the
    // first log2(kSortCap) stages stay inside them); every later stage runs its
    // long-distance steps in global memory and finishes each chunk in shared.
    const unsigned lgC = ceil_log2((unsigned)kSortCap);
    for (unsigned c0 = 0; c0 < n; c0 += kSortCap) {
        const unsigned m = min((unsigned)kSortCap, n - c0);
        for (unsigned i = threadIdx.x; i < (unsigned)kSortCap; i += blockDim.x) s_k[i] = i < m ? g[c0 + i] : kInfKey;
        __syncthreads();
        sort_pow2_smem(s_k, lgC);
        for (unsigned i = threadIdx.x; i < m; i += blockDim.x) g[c0 + i] = s_k[i];
        __syncthreads();
    }
    const unsigned lgN = ceil_log2(n), N = 1u << lgN;
    for (unsigned ls = lgC + 1; ls <= lgN; ++ls) {
        const unsigned lh = ls - 1, half = 1u << lh;
        for (unsigned tt = threadIdx.x; tt < (N >> 1); tt += blockDim.x) {
            const unsigned blk = tt >> lh, off = tt & (half - 1);
            const unsigned i = (blk << ls) + off, j = (blk << ls) + (1u << ls) - 1 - off;
            if (j < n) cswap(g, i, j);
        }
        __syncthreads();
        for (int ld = (int)ls - 2; ld >= (int)lgC; --ld) {
            const unsigned d = 1u << ld;
            for (unsigned tt = threadIdx.x; tt < (N >> 1); tt += blockDim.x) {
                const unsigned i = ((tt >> ld) << (ld + 1)) + (tt & (d - 1)), j = i + d;
                if (j < n) cswap(g, i, j);
            }
            __syncthreads();
        }
        // remaining cleaner steps (d < kSortCap) stay inside aligned chunks
        for (unsigned c0 = 0; c0 < n; c0 += kSortCap) {
            const unsigned m = min((unsigned)kSortCap, n - c0);
            for (unsigned i = threadIdx.x; i < (unsigned)kSortCap; i += blockDim.x) s_k[i] = i < m ? g[c0 + i] : kInfKey;
            __syncthreads();
            for (int ld = (int)lgC - 1; ld >= 6; --ld) {
                const unsigned d = 1u << ld;
                for (unsigned tt = threadIdx.x; tt < (unsigned)kSortCap / 2; tt += blockDim.x) {
                    const unsigned i = ((tt >> ld) << (ld + 1)) + (tt & (d - 1));
                    cswap(s_k, i, i + d);
                }
                __syncthreads();
            }
            const unsigned warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
            for (unsigned b = warp; b < (unsigned)kSortCap / 64; b += nw) {
                unsigned long long x0 = s_k[(b << 6) + 2 * lane], x1 = s_k[(b << 6) + 2 * lane + 1];
                reg_cleaners(x0, x1);
                s_k[(b << 6) + 2 * lane] = x0;
                s_k[(b << 6) + 2 * lane + 1] = x1;
            }
            __syncthreads();
            for (unsigned i = threadIdx.x; i < m; i += blockDim.x) g[c0 + i] = s_k[i];
            __syncthreads();
        }
    }
}

// In-place sort of a shared-memory segment k[0, n), 64 < n, by the whole block
// (call uniformly). Positions past n are virtual +inf keys: register blocks pad
// with +inf and write back only real keys; shared-memory comparators past n are
// skipped.
__device__ void sort_segment_smem(unsigned long long *k, unsigned n) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned lgN = ceil_log2(n), N = 1u << lgN, nblk = (n + 63) >> 6;
    for (unsigned b = warp; b < nblk; b += nw) {
        const unsigned i0 = (b << 6) + 2 * lane;
        unsigned long long x0 = i0 < n ? k[i0] : kInfKey, x1 = i0 + 1 < n ? k[i0 + 1] : kInfKey;
        reg_stages(x0, x1, 6);
        if (i0 < n) k[i0] = x0;
        if (i0 + 1 < n) k[i0 + 1] = x1;
    }
    __syncthreads();
    for (unsigned ls = 7; ls <= lgN; ++ls) {
        const unsigned lh = ls - 1, half = 1u << lh;
        for (unsigned t = threadIdx.x; t < (N >> 1); t += blockDim.x) {
            const unsigned blk = t >> lh, off = t & (half - 1);
            const unsigned i = (blk << ls) + off, j = (blk << ls) + (1u << ls) - 1 - off;
            if (j < n) cswap(k, i, j);
        }
        __syncthreads();
        for (int ld = (int)ls - 2; ld >= 6; --ld) {
            const unsigned d = 1u << ld;
            for (unsigned t = threadIdx.x; t < (N >> 1); t += blockDim.x) {
                const unsigned i = ((t >> ld) << (ld + 1)) + (t & (d - 1)), j = i + d;
                if (j < n) cswap(k, i, j);
            }
            __syncthreads();
        }
        for (unsigned b = warp; b < nblk; b += nw) {
            const unsigned i0 = (b << 6) + 2 * lane;
            unsigned long long x0 = i0 < n ? k[i0] : kInfKey, x1 = i0 + 1 < n ? k[i0 + 1] : kInfKey;
            reg_cleaners(x0, x1);
            if (i0 < n) k[i0] = x0;
            if (i0 + 1 < n) k[i0 + 1] = x1;
        }
        __syncthreads();
    }
}

// Refinement of a tile's depth buckets: a bucket of n_b > q keys is split by
// the next r_b = ceil(log2(ceil(n_b / q))) bits of the depth below its bin into
// 2^r_b sub-bins (the two clamped end bins, whose keys may span several
// exponents, are never split). 2^r_b < 2 n_b / q for a split bucket, so a tile
// of n keys has fewer than kDepthBins + 2 n / q sub-bins: q = kSubKeys keeps a
// tile of up to kSortCap keys within kMaxSub, and heavier tiles take
// q = ceil(2 n / (kMaxSub - kDepthBins)). Keys of a lower sub-bin precede those
// of a higher one, as keys of a lower bin precede those of a higher bin.
constexpr unsigned kSubKeys = 8;
constexpr int kMaxSub = kDepthBins + 2 * kSortCap / (int)kSubKeys;
constexpr int kSubPerThread = kMaxSub / kSortThreads;
static_assert(kMaxSub % kSortThreads == 0, "sub-bins are scanned kSubPerThread per thread");

__device__ __forceinline__ unsigned sub_bin(unsigned zb, const unsigned short *s_sb, const unsigned char *s_r) {
    const unsigned b = (unsigned)depth_bin(__uint_as_float(zb));
    return s_sb[b] + ((zb & 0x7ffffu) >> (19u - s_r[b]));
}

// One CTA per tile. The tile's keys are counted into refined depth sub-bins and
// scattered by sub-bin - into shared memory for a tile of up to kSortCap keys,
// else straight into the tile's range of the output list - and the sub-bins,
// merged into segments, are sorted: up to 128 keys by single warps in
// registers, longer ones by the whole block. A staged tile is stored back with
// one coalesced store.
// Fast path for a tile whose buckets all hold at most 32 keys (the common case when
// Gaussians are small): warp w takes buckets 32w .. 32w + 31 and walks them in windows
// of whole buckets of at most 32 keys. Keys of an earlier bucket precede those of a
// later one (the bucket is the depth bin, a monotone function of the depth bits that
// lead the key), so a key's place is its bucket's first place in the window plus the
// number of smaller keys in its bucket; the lanes of a bucket are found with match_any
// and compared with shuffles, one round per key of the largest bucket in the window.
// Keys go from the emission buffer to the sorted list directly.
__device__ __forceinline__ unsigned key_bin(unsigned long long key) {
    const int b = (int)((unsigned)(key >> 32) >> 19) - 1993;  // depth_bin of the key's depth bits
    return b < 0 ? 0u : (b > kDepthBins - 1 ? (unsigned)(kDepthBins - 1) : (unsigned)b);
}

__device__ void sort_small_buckets(const SortArgs &a, const unsigned *bs, unsigned base) {
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const unsigned long long *in = a.keys_in + base;
    unsigned long long *out = a.keys + base;
    const unsigned bnd = bs[32 * w + lane] - base;  // start of bucket 32 w + lane
    const unsigned endw = bs[32 * w + 32] - base;
    unsigned w0 = __shfl_sync(0xffffffffu, bnd, 0);
    while (w0 < endw) {
        // the window ends at the last bucket boundary within 32 keys (every bucket is
        // at most 32 keys long, so there is one beyond w0)
        const unsigned lim = w0 + 32u;
        const unsigned w1 = max(__reduce_max_sync(0xffffffffu, (bnd > w0 && bnd <= lim) ? bnd : 0u),
                                endw <= lim ? endw : 0u);
        const unsigned i = w0 + lane;
        const bool act = i < w1;
        const unsigned long long key = act ? in[i] : kInfKey;
        const unsigned peers = __match_any_sync(0xffffffffu, act ? key_bin(key) : 0x10000u + lane);
        const unsigned first = __ffs(peers) - 1, size = __popc(peers);
        const unsigned rounds = __reduce_max_sync(0xffffffffu, act ? size : 0u);
        unsigned rank = 0;
        for (unsigned d = 0; d < rounds; ++d) {
            const unsigned long long y = __shfl_sync(0xffffffffu, key, (first + d) & 31u);
            rank += (d < size && y < key) ? 1u : 0u;
        }
        if (act) out[w0 + first + rank] = key;
        if (w1 <= w0) break;  // cannot happen: the caller checked every bucket's length
        w0 = w1;
    }
}

__global__ void __launch_bounds__(kSortThreads, 5) tile_sort_kernel(const SortArgs a) {
    __shared__ unsigned long long s_k[kSortCap];
    __shared__ unsigned s_start[kDepthBins + 1];
    __shared__ unsigned s_seg[kMaxSub + 1];        // sub-bin cursors, then segment starts
    __shared__ unsigned s_sub[kMaxSub + 1];        // sub-bin starts
    __shared__ unsigned short s_sb[kDepthBins];    // first sub-bin of each bucket
    __shared__ unsigned char s_r[kDepthBins];      // refinement bits of each bucket
    __shared__ unsigned s_warp[33];
    if (a.ctr->overflow) return;
    const long long t = blockIdx.x;
    const unsigned *bs = a.tile_start + t * kDepthBins;
    const unsigned base = bs[0], n_tile = bs[kDepthBins] - base;
    const unsigned long long *in = a.keys_in + base;
    if (n_tile <= 1) {
        if (n_tile == 1 && threadIdx.x == 0) a.keys[base] = in[0];
        return;
    }
    static_assert(kSortThreads == kDepthBins, "one thread per bucket");
    const unsigned b = threadIdx.x;
    if (!__syncthreads_or(bs[b + 1] - bs[b] > 32u)) {
        sort_small_buckets(a, bs, base);
        return;
    }
    s_start[b] = bs[b] - base;
    if (b == 0) s_start[kDepthBins] = n_tile;
    __syncthreads();
    const bool staged = n_tile <= (unsigned)kSortCap;
    unsigned long long *keys = staged ? s_k : a.keys + base;
    constexpr unsigned long long kSplit = kMaxSub - kDepthBins;
    const unsigned q = staged ? kSubKeys
                              : max(kSubKeys, (unsigned)((2ull * n_tile + kSplit - 1) / kSplit));
    const unsigned nb = s_start[b + 1] - s_start[b];
    const unsigned r = (b == 0 || b == kDepthBins - 1 || nb <= q)
                           ? 0u : ceil_log2((unsigned)(((unsigned long long)nb + q - 1) / q));
    unsigned n_sub;
    s_sb[b] = (unsigned short)block_excl_scan(1u << r, s_warp, &n_sub);
    s_r[b] = (unsigned char)r;
    for (unsigned j = threadIdx.x; j < n_sub; j += blockDim.x) s_seg[j] = 0;
    __syncthreads();
    // both passes over the tile's keys keep four loads in flight per thread
    for (unsigned i0 = threadIdx.x; i0 < n_tile; i0 += 4 * blockDim.x) {
        unsigned zb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned i = i0 + u * blockDim.x;
            zb[u] = i < n_tile ? (unsigned)(in[i] >> 32) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u * blockDim.x < n_tile) atomicAdd(&s_seg[sub_bin(zb[u], s_sb, s_r)], 1u);
    }
    __syncthreads();
    unsigned c[kSubPerThread], sum = 0, tot;
#pragma unroll
    for (int k = 0; k < kSubPerThread; ++k) {
        const unsigned j = kSubPerThread * b + k;
        c[k] = j < n_sub ? s_seg[j] : 0u;
        sum += c[k];
    }
    unsigned ex = block_excl_scan(sum, s_warp, &tot);
#pragma unroll
    for (int k = 0; k < kSubPerThread; ++k) {
        const unsigned j = kSubPerThread * b + k;
        if (j < n_sub) {
            s_sub[j] = ex;
            s_seg[j] = ex;
        }
        ex += c[k];
    }
    if (b == 0) s_sub[n_sub] = n_tile;
    __syncthreads();
    for (unsigned i0 = threadIdx.x; i0 < n_tile; i0 += 4 * blockDim.x) {
        unsigned long long key[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned i = i0 + u * blockDim.x;
            key[u] = i < n_tile ? in[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u * blockDim.x < n_tile)
                keys[atomicAdd(&s_seg[sub_bin((unsigned)(key[u] >> 32), s_sb, s_r)], 1u)] = key[u];
    }
    __syncthreads();
    // Merge consecutive sub-bins into segments: a new segment starts at the
    // first sub-bin beginning in each window of kSegKeys keys. Keys of an
    // earlier sub-bin all precede those of a later one, so sorting a segment as
    // a whole equals sorting its sub-bins one by one; segments hold about
    // kSegKeys keys, which keeps the warps' register sorts full.
    unsigned f = 0, fl[kSubPerThread], n_seg;
#pragma unroll
    for (int k = 0; k < kSubPerThread; ++k) {
        const unsigned j = kSubPerThread * b + k;
        fl[k] = j < n_sub && (j == 0 || s_sub[j] / kSegKeys != s_sub[j - 1] / kSegKeys);
        f += fl[k];
    }
    unsigned idx = block_excl_scan(f, s_warp, &n_seg);
#pragma unroll
    for (int k = 0; k < kSubPerThread; ++k)
        if (fl[k]) s_seg[idx++] = s_sub[kSubPerThread * b + k];
    if (b == 0) s_seg[n_seg] = n_tile;
    __syncthreads();
    const unsigned warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    bool any_large = false;
    for (unsigned i = warp; i < n_seg; i += nw) {
        const unsigned n = s_seg[i + 1] - s_seg[i];
        if (n < 2) continue;
        if (n <= 128) sort_segment_warp(keys + s_seg[i], n);
        else any_large = true;
    }
    if (__syncthreads_or(any_large)) {
        for (unsigned i = 0; i < n_seg; ++i) {
            const unsigned n = s_seg[i + 1] - s_seg[i];
            if (n <= 128) continue;
            if (staged) sort_segment_smem(s_k + s_seg[i], n);
            else sort_segment_block(a.keys + base + s_seg[i], n, s_k);
        }
    }
    if (staged) {
        __syncthreads();
        for (unsigned i = threadIdx.x; i < n_tile; i += blockDim.x) a.keys[base + i] = s_k[i];
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
        atomicAdd(&s_c[load_bucket(a.tile_start[(t + 1) * kDepthBins] - a.tile_start[t * kDepthBins])], 1u);
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
        int b = load_bucket(a.tile_start[(t + 1) * kDepthBins] - a.tile_start[t * kDepthBins]);
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
    if (vb.n_views == 0 || a.n == 0) return cudaSuccess;
    emit_kernel<false><<<dim3((unsigned)((a.n + 255) / 256), (unsigned)vb.n_views), 256, 0, s>>>(a, vb);
    return cudaGetLastError();
}

cudaError_t launch_count(const EmitArgs &a, const ViewBatch &vb, cudaStream_t s) {
    if (vb.n_views == 0 || a.n == 0) return cudaSuccess;
    emit_kernel<true><<<dim3((unsigned)((a.n + 255) / 256), (unsigned)vb.n_views), 256, 0, s>>>(a, vb);
    return cudaGetLastError();
}

cudaError_t launch_cut(const CutArgs &a, const ViewBatch &vb, cudaStream_t s) {
    if (a.n_tiles == 0) return cudaSuccess;
    cut_kernel<<<(unsigned)((a.n_tiles + 7) / 8), 256, 0, s>>>(a, vb);
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
