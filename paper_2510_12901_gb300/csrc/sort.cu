// sort.cu -- binning and the (tile, depth) key sort (the "Sort" kernel of
// the paper's App. B timing table; keys as in 3DGS, Sec. 3.2).
//
// Order of work (all on the device, one 4-byte read-back of the pair count):
//   1. compact the Gaussians that survived projection into (depth bits, id)
//      pairs, in id order;
//   2. stable LSD radix sort of those pairs by depth (4 passes of 8 bits):
//      ties keep id order, so the order is (depth, id);
//   3. gather tile counts in that order and scan them into pair offsets;
//   4. bin: every Gaussian writes (tile, id) for each tile of its range, so
//      the pair list is in (depth, id) order;
//   5. stable LSD radix sort of the pairs by tile id only (2 passes for up
//      to 65536 tiles), which yields (tile, depth, id) order;
//   6. per-tile [start, end) ranges.
// Sorting the N Gaussians by depth once and the K pairs by tile alone moves
// 2 passes over K instead of the 6 a 64-bit (tile, depth) key needs.
#include "internal.h"

namespace sg {

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t *total)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (lane < nw) s_warp[lane] = wi - w;
        if (lane == nw - 1) s_warp[32] = wi;
    }
    __syncthreads();
    uint32_t r = s_warp[warp] + inc - v;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ part)
{
    __shared__ uint32_t s_warp[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) acc += in[idx];
    }
    uint32_t tot;
    block_excl_scan(acc, s_warp, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Exclusive scan of one tile per block, offset by the scanned partials.
__global__ void __launch_bounds__(kScanThreads)
k_scan_down(const uint32_t *__restrict__ in, int64_t n, const uint32_t *__restrict__ part_scanned,
            uint32_t *__restrict__ out, uint32_t *__restrict__ total)
{
    __shared__ uint32_t s_val[kScanTile];
    __shared__ uint32_t s_warp[33];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        s_val[i * kScanThreads + threadIdx.x] = idx < n ? in[idx] : 0u;
    }
    __syncthreads();
    uint32_t loc[kScanItems], acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        loc[i] = acc;
        acc += s_val[threadIdx.x * kScanItems + i];
    }
    uint32_t tot;
    uint32_t pre = block_excl_scan(acc, s_warp, &tot) + (part_scanned ? part_scanned[blockIdx.x] : 0u);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) s_val[threadIdx.x * kScanItems + i] = pre + loc[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) out[idx] = s_val[i * kScanThreads + threadIdx.x];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        // the grand total = scanned offset of this last tile + its sum
        *total = (part_scanned ? part_scanned[blockIdx.x] : 0u) + tot;
    }
}

// Exclusive scan; scratch comes from fr.scan_tmp (grown as needed).  The
// partial sums are scanned recursively with the same two kernels.
static sg_status scan_rec(const uint32_t *in, uint32_t *out, uint32_t *total, int64_t n,
                          uint32_t *scratch, cudaStream_t st)
{
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= 1) {
        k_scan_down<<<1, kScanThreads, 0, st>>>(in, n, nullptr, out, total);
        SG_LAUNCHED();
        return SG_OK;
    }
    uint32_t *part = scratch, *part_scanned = scratch + nb;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, part);
    SG_LAUNCHED();
    sg_status s = scan_rec(part, part_scanned, nullptr, nb, scratch + 2 * nb, st);
    if (s != SG_OK) return s;
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, part_scanned, out, total);
    SG_LAUNCHED();
    return SG_OK;
}

static int64_t scan_scratch_words(int64_t n)
{
    int64_t w = 0;
    while (true) {
        int64_t nb = (n + kScanTile - 1) / kScanTile;
        if (nb <= 1) break;
        w += 2 * nb;
        n = nb;
    }
    return w + 16;
}

sg_status scan_exclusive_u32(const uint32_t *d_in, uint32_t *d_out, uint32_t *d_total,
                             int64_t n, Frame &fr, cudaStream_t st)
{
    if (n <= 0) {
        if (d_total) SG_CUDA(cudaMemsetAsync(d_total, 0, 4, st));
        return SG_OK;
    }
    sg_status s = ensure(fr.scan_tmp, sizeof(uint32_t) * scan_scratch_words(n));
    if (s != SG_OK) return s;
    return scan_rec(d_in, d_out, d_total, n, (uint32_t *)fr.scan_tmp.p, st);
}

// ------------------------------------------------------------------ radix sort
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;   // 2048
constexpr int kRadixWarps = kRadixThreads / 32;

// Per-block digit histogram, stored digit-major (hist[d * nblocks + b]) so
// that one exclusive scan over it yields every block's output offsets.
__global__ void __launch_bounds__(kRadixThreads)
k_radix_hist(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ d_n, int shift,
             uint32_t mask, uint32_t *__restrict__ hist, int nblocks)
{
    __shared__ uint32_t s_h[256];
    s_h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t n = *d_n;
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (base < n) {
#pragma unroll
        for (int r = 0; r < kRadixItems; ++r) {
            int64_t idx = base + (int64_t)warp * 32 * kRadixItems + r * 32 + lane;
            bool in = idx < n;
            uint32_t d = in ? (keys[idx] >> shift) & mask : 0xffffffffu;
            uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (in && lane == __ffs(peers) - 1) atomicAdd(&s_h[d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter: warp w owns elements [w*256, (w+1)*256) of the block tile,
// taken 32 at a time in order; ranks among equal digits come from
// __match_any_sync, warp offsets from a per-digit scan over the warps.
__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                const uint32_t *__restrict__ d_n, int shift, uint32_t mask,
                const uint32_t *__restrict__ hist_scanned, int nblocks)
{
    __shared__ uint32_t s_cnt[kRadixWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRadixWarps * 256; i += kRadixThreads) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = *d_n;
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    if (base >= n) return;
    uint32_t k[kRadixItems], v[kRadixItems], d[kRadixItems], rk[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        int64_t idx = base + (int64_t)warp * 32 * kRadixItems + r * 32 + lane;
        bool in = idx < n;
        k[r] = in ? keys_in[idx] : 0u;
        v[r] = in ? vals_in[idx] : 0u;
        d[r] = in ? (k[r] >> shift) & mask : 0xffffffffu;
        uint32_t peers = __match_any_sync(0xffffffffu, d[r]);
        uint32_t below = __popc(peers & ((1u << lane) - 1u));
        uint32_t before = in ? s_cnt[warp][d[r]] : 0u;
        rk[r] = before + below;
        __syncwarp();
        if (in && lane == __ffs(peers) - 1) s_cnt[warp][d[r]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, plus the global offset
    {
        uint32_t dgt = threadIdx.x;   // 256 threads, one digit each
        uint32_t run = hist_scanned[(int64_t)dgt * nblocks + blockIdx.x];
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) {
            uint32_t c = s_cnt[w][dgt];
            s_cnt[w][dgt] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        int64_t idx = base + (int64_t)warp * 32 * kRadixItems + r * 32 + lane;
        if (idx < n) {
            uint32_t pos = s_cnt[warp][d[r]] + rk[r];
            keys_out[pos] = k[r];
            vals_out[pos] = v[r];
        }
    }
}

sg_status radix_sort_pairs(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max,
                           const uint32_t *d_n, int begin_bit, int end_bit, Frame &fr,
                           cudaStream_t st, int *result_buf)
{
    int cur = 0;
    *result_buf = 0;
    if (n_max <= 0 || end_bit <= begin_bit) return SG_OK;
    int nblocks = (int)((n_max + kRadixTile - 1) / kRadixTile);
    int64_t nh = (int64_t)nblocks * 256;
    sg_status s = ensure(fr.hist, sizeof(uint32_t) * 2 * nh);
    if (s != SG_OK) return s;
    uint32_t *hist = (uint32_t *)fr.hist.p, *hist_sc = hist + nh;
    for (int b = begin_bit; b < end_bit; b += 8) {
        int bits = end_bit - b < 8 ? end_bit - b : 8;
        uint32_t mask = (1u << bits) - 1u;
        k_radix_hist<<<nblocks, kRadixThreads, 0, st>>>(keys[cur], d_n, b, mask, hist, nblocks);
        SG_LAUNCHED();
        s = scan_exclusive_u32(hist, hist_sc, nullptr, nh, fr, st);
        if (s != SG_OK) return s;
        k_radix_scatter<<<nblocks, kRadixThreads, 0, st>>>(keys[cur], vals[cur], keys[cur ^ 1],
                                                           vals[cur ^ 1], d_n, b, mask, hist_sc,
                                                           nblocks);
        SG_LAUNCHED();
        cur ^= 1;
    }
    *result_buf = cur;
    return SG_OK;
}

// ------------------------------------------------------------------ compaction

__global__ void k_flags(const uint32_t *__restrict__ count, int64_t n, uint32_t *__restrict__ flags)
{
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) flags[g] = count[g] > 0 ? 1u : 0u;
}

__global__ void k_compact(const uint32_t *__restrict__ count, const float *__restrict__ depth,
                          const uint32_t *__restrict__ pos, int64_t n, uint32_t *__restrict__ keys,
                          uint32_t *__restrict__ vals)
{
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n && count[g] > 0) {
        uint32_t p = pos[g];
        keys[p] = __float_as_uint(depth[g]);   // depth > 0: bits are monotone
        vals[p] = (uint32_t)g;
    }
}

sg_status compact_valid(const uint32_t *d_count, const float *d_depth, int64_t n,
                        uint32_t *d_keys, uint32_t *d_vals, uint32_t *d_nvalid, Frame &fr,
                        cudaStream_t st)
{
    if (n == 0) {
        SG_CUDA(cudaMemsetAsync(d_nvalid, 0, 4, st));
        return SG_OK;
    }
    sg_status s = ensure(fr.flags, sizeof(uint32_t) * 2 * n);
    if (s != SG_OK) return s;
    uint32_t *flags = (uint32_t *)fr.flags.p, *pos = flags + n;
    unsigned grid = (unsigned)((n + 255) / 256);
    k_flags<<<grid, 256, 0, st>>>(d_count, n, flags);
    SG_LAUNCHED();
    s = scan_exclusive_u32(flags, pos, d_nvalid, n, fr, st);
    if (s != SG_OK) return s;
    k_compact<<<grid, 256, 0, st>>>(d_count, d_depth, pos, n, d_keys, d_vals);
    SG_LAUNCHED();
    return SG_OK;
}

__global__ void k_gather_counts(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ count,
                                const uint32_t *__restrict__ d_nvalid, int64_t n,
                                uint32_t *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = i < (int64_t)*d_nvalid ? count[ids[i]] : 0u;
}

sg_status gather_counts(const uint32_t *d_ids, const uint32_t *d_count, const uint32_t *d_nvalid,
                        int64_t n, uint32_t *d_out, cudaStream_t st)
{
    if (n == 0) return SG_OK;
    k_gather_counts<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_ids, d_count, d_nvalid, n,
                                                                 d_out);
    SG_LAUNCHED();
    return SG_OK;
}

// ------------------------------------------------------------------ binning

// Expand each valid Gaussian (depth order) into its (tile, Gaussian) pairs:
// pair o of Gaussian g goes to position offsets[g] + o, tile rows outer and
// columns inner.  A block takes 256 consecutive Gaussians and writes all of
// their pairs with its threads striding over the output positions (the
// owner of a position is found by binary search over the block's offsets),
// so a Gaussian that covers many tiles does not serialise one thread and
// the writes are coalesced.  Pairs at positions >= cap are not written
// (capacity mode: the caller learns of them from the dropped-pairs count).
constexpr int kBinThreads = 256;

__global__ void __launch_bounds__(kBinThreads)
k_bin(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offsets,
      const uint32_t *__restrict__ counts, const uint32_t *__restrict__ d_nvalid,
      const int4 *__restrict__ tiles, int ntx, int wrap_x, uint32_t cap,
      uint32_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    __shared__ uint32_t s_off[kBinThreads], s_id[kBinThreads];
    __shared__ int4 s_rect[kBinThreads];
    __shared__ uint32_t s_end;
    const int64_t g0 = (int64_t)blockIdx.x * kBinThreads;
    const int64_t nvalid = *d_nvalid;
    if (g0 >= nvalid) return;
    const int nb = (int)min((int64_t)kBinThreads, nvalid - g0);
    const int t = threadIdx.x;
    if (t < nb) {
        const uint32_t g = ids[g0 + t];
        s_id[t] = g;
        s_off[t] = offsets[g0 + t];
        s_rect[t] = tiles[g];
        if (t == nb - 1) s_end = offsets[g0 + t] + counts[g0 + t];
    }
    __syncthreads();
    const uint32_t first = s_off[0], total = s_end - first;
    for (uint32_t o = t; o < total; o += kBinThreads) {
        const uint32_t pos = first + o;
        int lo = 0, hi = nb;      // owner: the last k with s_off[k] <= pos
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= pos) lo = mid; else hi = mid;
        }
        if (pos >= cap) continue;
        const int4 r = s_rect[lo];
        const uint32_t local = pos - s_off[lo], w = (uint32_t)(r.y - r.x + 1);
        const int ty = r.z + (int)(local / w);
        int x = r.x + (int)(local % w);
        if (wrap_x) { x %= ntx; if (x < 0) x += ntx; }
        keys[pos] = (uint32_t)(ty * ntx + x);
        vals[pos] = s_id[lo];
    }
}

sg_status bin_pairs(const uint32_t *d_ids, const uint32_t *d_offsets, const uint32_t *d_counts,
                    const uint32_t *d_nvalid, int64_t n, const int4 *d_tiles, int ntx, int wrap_x,
                    int64_t cap, uint32_t *d_keys, uint32_t *d_vals, cudaStream_t st)
{
    if (n == 0) return SG_OK;
    k_bin<<<(unsigned)((n + kBinThreads - 1) / kBinThreads), kBinThreads, 0, st>>>(
        d_ids, d_offsets, d_counts, d_nvalid, d_tiles, ntx, wrap_x, (uint32_t)cap, d_keys, d_vals);
    SG_LAUNCHED();
    return SG_OK;
}

__global__ void k_ranges(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ d_K,
                         uint2 *__restrict__ ranges)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t K = *d_K;
    if (i >= K) return;
    uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == K - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
}

sg_status tile_ranges(const uint32_t *d_keys, const uint32_t *d_K, int64_t K_max, uint2 *d_ranges,
                      int64_t ntiles, cudaStream_t st)
{
    SG_CUDA(cudaMemsetAsync(d_ranges, 0, sizeof(uint2) * ntiles, st));
    if (K_max == 0) return SG_OK;
    k_ranges<<<(unsigned)((K_max + 255) / 256), 256, 0, st>>>(d_keys, d_K, d_ranges);
    SG_LAUNCHED();
    return SG_OK;
}

// Capacity mode: keep at most `cap` pairs; d_K is clamped to it and the
// number of pairs beyond it is stored in d_dropped (0 when all fit).
__global__ void k_clamp_pairs(uint32_t *__restrict__ d_K, uint32_t cap,
                              uint32_t *__restrict__ d_dropped)
{
    const uint32_t K = *d_K;
    *d_dropped = K > cap ? K - cap : 0u;
    if (K > cap) *d_K = cap;
}

sg_status clamp_pairs(uint32_t *d_K, int64_t cap, uint32_t *d_dropped, cudaStream_t st)
{
    k_clamp_pairs<<<1, 1, 0, st>>>(d_K, (uint32_t)cap, d_dropped);
    SG_LAUNCHED();
    return SG_OK;
}

}  // namespace sg
