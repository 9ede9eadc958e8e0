// sort.cu -- binning and the (tile, depth) key sort (the "Sort" kernel of
// the paper's App. B timing table; keys as in 3DGS, Sec. 3.2).
//
// Order of work (all on the device, one 4-byte read-back of the pair count):
//   1. compact the Gaussians that survived projection into (depth bits, id)
//      pairs, in id order, counting the radix digits as it goes;
//   2. stable LSD radix sort of those pairs by depth (4 passes of 8 bits):
//      ties keep id order, so the order is (depth, id);
//   3. scan their tile counts, in that order, into pair offsets;
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

// ------------------------------------------------------------------ radix sort
// Lanes of the warp holding the same 8-bit digit as this one, among lanes
// with a key (valid): one ballot per bit, each lane keeping the lanes that
// agree with it on that bit.  A lane without a key is in no lane's set.
// (Nine ballots take less time here than __match_any_sync: the depth stage
// went from 0.144 to 0.127 ms per view.)
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid)
{
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bb = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bb : ~bb;
    }
    return peers;
}

// Stable LSD radix sort of (key, value) pairs, 8-bit digits, one kernel per
// digit pass with decoupled look-back (the "onesweep" scheme):
//   1. the kernel that writes the keys counts the digits of every pass
//      (k_compact_depth, k_bin) into scratch that radix_prepare zeroed;
//   2. per pass, the exclusive scan of its 256 counts gives the first
//      output position of each digit (every block of the pass scans them);
//   3. k_onesweep, per pass: a block takes the next tile of kRadixTile pairs
//      (an atomic ticket, so tiles are taken in order), ranks them stably
//      (each warp owns kRadixItems x 32 consecutive pairs, ranks among equal
//      digits from per-bit ballots), publishes its per-digit counts, and
//      walks back over earlier tiles' published counts, kLbBatch tiles per
//      round of loads, until it meets an inclusive prefix; then it
//      publishes its own inclusive prefix and scatters.
// A tile only waits for tiles taken before it, whose blocks are running;
// every such wait is bounded, and a wait that runs out sets *err.
#ifndef SG_RADIX_THREADS
#define SG_RADIX_THREADS 1024
#endif
constexpr int kRadixThreads = SG_RADIX_THREADS;   // >= 256: one digit per thread below 256
constexpr int kRadixItems = kRadixTile / kRadixThreads;
static_assert(kRadixThreads >= 256 && kRadixItems * kRadixThreads == kRadixTile,
              "radix tile layout");
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr uint32_t kLbAgg = 1u << 30, kLbPre = 2u << 30, kLbCount = (1u << 30) - 1u;
// Polling rounds a look-back wait makes before it gives up (about a second
// on an idle GPU).  Test hook: the tile whose look-back words the kernels
// of one site never publish (-1: none), so that the next tile's wait runs
// out.  Both live in device memory, where sg_debug_lookback sets them, so
// that replays of captured launch sequences see them too.
constexpr uint32_t kLbSpinsDefault = 1u << 20;
__device__ uint32_t g_lb_spins = kLbSpinsDefault;
__device__ int g_hold_site = SG_LOOKBACK_NONE;
__device__ long long g_hold_tile = -1;
// The tile this launch (of `site`) withholds, or -1.
__device__ __forceinline__ int64_t held_tile(int site)
{
    return *(volatile int *)&g_hold_site == site ? (int64_t) * (volatile long long *)&g_hold_tile
                                                 : (int64_t)-1;
}
#ifndef SG_LB_BATCH
#define SG_LB_BATCH 8
#endif
constexpr int kLbBatch = SG_LB_BATCH;   // earlier tiles' words loaded per look-back round

__global__ void __launch_bounds__(kRadixThreads)
k_onesweep(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
           uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
           const uint32_t *__restrict__ d_n, int shift, uint32_t mask,
           const uint32_t *__restrict__ hist, uint32_t *__restrict__ lookback,
           uint32_t *__restrict__ ticket, uint32_t *__restrict__ err, int site)
{
    __shared__ uint32_t s_cnt[kRadixWarps][256];
    __shared__ uint32_t s_pre[256];
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRadixWarps * 256; i += kRadixThreads) (&s_cnt[0][0])[i] = 0;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t n = *d_n;
    const int64_t base = (int64_t)tile * kRadixTile;
    if (base >= n) return;     // so is every later tile: nobody waits for this one
    // the first output position of this thread's digit (threads < 256): the
    // exclusive scan of the pass's digit counts, done by every block
    uint32_t dig_total;
    const uint32_t dig_off =
        block_excl_scan(threadIdx.x < 256 ? hist[threadIdx.x] : 0u, s_warp, &dig_total);
    uint32_t k[kRadixItems], v[kRadixItems], d[kRadixItems], rk[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const int64_t idx = base + (int64_t)warp * 32 * kRadixItems + r * 32 + lane;
        const bool in = idx < n;
        k[r] = in ? keys_in[idx] : 0u;
        v[r] = in ? vals_in[idx] : 0u;
        d[r] = in ? (k[r] >> shift) & mask : 0xffffffffu;
        const uint32_t peers = digit_peers(d[r], in);
        const uint32_t below = __popc(peers & ((1u << lane) - 1u));
        const uint32_t before = in ? s_cnt[warp][d[r]] : 0u;
        rk[r] = before + below;
        __syncwarp();
        if (in && lane == __ffs(peers) - 1) s_cnt[warp][d[r]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < 256) {
        // one digit per thread: offsets of the warps within the tile, the
        // tile's count, then the look-back for the pairs of earlier tiles
        const uint32_t dg = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) {
            const uint32_t c = s_cnt[w][dg];
            s_cnt[w][dg] = run;
            run += c;
        }
        volatile uint32_t *lb = lookback;
        const bool publish = (int64_t)tile != held_tile(site);
        const uint32_t max_spins = g_lb_spins;
        if (publish) lb[(int64_t)tile * 256 + dg] = (tile == 0 ? kLbPre : kLbAgg) | run;
        uint32_t excl = 0, spins = 0;
        int64_t t = (int64_t)tile - 1;
        while (t >= 0) {
            // the words of tiles t, t-1, .. at once (before tile 0: an empty
            // inclusive prefix); take them in order up to an inclusive prefix
            // or up to one not yet published, which the next round reloads
            uint32_t w[kLbBatch];
#pragma unroll
            for (int k = 0; k < kLbBatch; ++k)
                w[k] = t - k >= 0 ? (uint32_t)lb[(t - k) * 256 + dg] : (uint32_t)kLbPre;
            int took = 0;
            bool pre = false, wait = false;
#pragma unroll
            for (int k = 0; k < kLbBatch; ++k) {
                if (pre || wait) continue;
                if (w[k] & (kLbAgg | kLbPre)) {
                    excl += w[k] & kLbCount;
                    pre = (w[k] & kLbPre) != 0u;
                    ++took;
                } else {
                    wait = true;
                }
            }
            if (pre) break;
            t -= took;
            if (took == 0 && ++spins > max_spins) {   // gave up: flag it, leave the order wrong
                atomicOr(err, kStatusLookback);
                break;
            }
        }
        if (tile > 0 && publish) lb[(int64_t)tile * 256 + dg] = kLbPre | (excl + run);
        s_pre[dg] = dig_off + excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const int64_t idx = base + (int64_t)warp * 32 * kRadixItems + r * 32 + lane;
        if (idx < n) {
            const uint32_t pos = s_pre[d[r]] + s_cnt[warp][d[r]] + rk[r];
            keys_out[pos] = k[r];
            vals_out[pos] = v[r];
        }
    }
}

// Zero the radix scratch (histograms, tickets, look-back words) for a sort
// of up to n_max pairs in `passes` passes; *hist gets the histograms, which
// the kernel that writes the keys fills before radix_sort_pairs runs.
// `extra` more zeroed words follow the scratch (at hist + radix_scratch_words).
sg_status radix_prepare(int64_t n_max, int passes, Frame &fr, cudaStream_t st, uint32_t **hist,
                        int64_t extra)
{
    const int64_t words = radix_scratch_words(n_max, passes) + extra;
    sg_status s = ensure(fr.hist, sizeof(uint32_t) * words);
    if (s != SG_OK) return s;
    SG_CUDA(cudaMemsetAsync(fr.hist.p, 0, sizeof(uint32_t) * words, st));
    *hist = (uint32_t *)fr.hist.p;
    return SG_OK;
}

sg_status radix_sort_pairs(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max,
                           const uint32_t *d_n, int begin_bit, int end_bit, Frame &fr,
                           cudaStream_t st, int *result_buf, int site)
{
    *result_buf = 0;
    if (n_max <= 0 || end_bit <= begin_bit) return SG_OK;
    if (n_max > (int64_t)kLbCount) {
        set_error("radix sort of %lld pairs exceeds 2^30", (long long)n_max);
        return SG_ERR_OVERFLOW;
    }
    const int passes = (end_bit - begin_bit + 7) / 8;
    const int64_t tiles = (n_max + kRadixTile - 1) / kRadixTile;
    uint32_t *hist = (uint32_t *)fr.hist.p;
    uint32_t *tickets = hist + 2 * 256 * passes;            // [passes], padded to 16
    uint32_t *lookback = tickets + 16;
    uint32_t *err = (uint32_t *)fr.scalars.p + kScalStatus;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const int b = begin_bit + 8 * p;
        const int bits = end_bit - b < 8 ? end_bit - b : 8;
        k_onesweep<<<(unsigned)tiles, kRadixThreads, 0, st>>>(
            keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], d_n, b, (1u << bits) - 1u,
            hist + 256 * p, lookback + (int64_t)p * tiles * 256, tickets + p, err, site);
        SG_LAUNCHED();
        cur ^= 1;
    }
    *result_buf = cur;
    return SG_OK;
}

// ------------------------------------------------------------------ depth stage
// The depth stage as two chained scans around the radix passes.  A block
// takes the next tile of kChainTile entries (an atomic ticket, so tiles are
// taken in order), publishes its total, and walks back over earlier tiles'
// published totals until an inclusive prefix (64-bit words: two flag bits,
// a 62-bit count), as the radix passes do:
//   k_compact_depth: the Gaussians with a non-zero tile count, in id order,
//     as (depth bits, id) pairs, the number of them, and the digit
//     histograms of the four radix passes over their keys;
//   k_pair_offsets: in depth order, the exclusive scan of the tile counts
//     count[ids[i]] (gathered as it goes) into pair offsets, and the total.
constexpr int kChainThreads = 256;
constexpr int kChainWarps = kChainThreads / 32;
constexpr int kChainChunks = kChainTile / kChainThreads;   // 32-entry chunks per warp
static_assert(kChainChunks * kChainThreads == kChainTile && kChainChunks == 16, "chain tile");
constexpr unsigned long long kChAgg = 1ull << 62, kChPre = 2ull << 62,
                             kChCount = (1ull << 62) - 1ull;

// Exclusive prefix of tile `tile` (total `total`) from the earlier tiles'
// words, 32 of them per round; warp 0 runs it and every lane returns it.  A
// wait that runs out sets *err (the prefix is then wrong, never unbounded).
__device__ unsigned long long chain_lookback(unsigned long long *lb, int64_t tile,
                                             unsigned long long total, uint32_t *err, int site)
{
    const int lane = threadIdx.x & 31;
    volatile unsigned long long *v = lb;
    const bool publish = tile != held_tile(site);
    const uint32_t max_spins = g_lb_spins;
    if (lane == 0 && publish) v[tile] = (tile == 0 ? kChPre : kChAgg) | total;
    unsigned long long excl = 0;
    uint32_t spins = 0;
    int64_t t = tile - 1;
    while (t >= 0) {
        const int64_t tt = t - lane;
        const unsigned long long w = tt >= 0 ? v[tt] : (unsigned long long)kChPre;   // before tile 0: empty prefix
        const uint32_t np = __ballot_sync(0xffffffffu, (w & (kChAgg | kChPre)) == 0ull);
        const uint32_t pre = __ballot_sync(0xffffffffu, (w & kChPre) != 0ull);
        const int fnp = np ? __ffs(np) - 1 : 32, fp = pre ? __ffs(pre) - 1 : 32;
        const int take = fp < fnp ? fp + 1 : fnp;   // lanes [0, take) are summed
        unsigned long long c = lane < take ? (w & kChCount) : 0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        excl += c;
        if (fp < fnp) break;
        t -= take;
        if (take == 0 && ++spins > max_spins) {   // gave up: flag it
            if (lane == 0) atomicOr(err, kStatusLookback);
            break;
        }
    }
    if (lane == 0 && tile > 0 && publish) v[tile] = kChPre | (excl + total);
    return excl;
}

__global__ void __launch_bounds__(kChainThreads)
k_compact_depth(const uint32_t *__restrict__ count, const float *__restrict__ depth, int64_t n,
                int64_t ntiles, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                uint32_t *__restrict__ d_nvalid, uint32_t *__restrict__ hist,
                unsigned long long *__restrict__ lb, uint32_t *__restrict__ ticket,
                uint32_t *__restrict__ err)
{
    __shared__ uint32_t s_h[4][256];
    __shared__ uint32_t s_warp[kChainWarps];
    __shared__ uint32_t s_tile;
    for (int i = threadIdx.x; i < 4 * 256; i += kChainThreads) (&s_h[0][0])[i] = 0;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warp w owns kChainChunks x 32 consecutive entries of the tile
    const int64_t wbase = tile * kChainTile + (int64_t)warp * 32 * kChainChunks;
    uint32_t cnt[kChainChunks], bal[kChainChunks], key[kChainChunks];
#pragma unroll
    for (int r = 0; r < kChainChunks; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        cnt[r] = i < n ? count[i] : 0u;
        key[r] = i < n ? __float_as_uint(depth[i]) : 0u;   // depth > 0: bits are monotone
    }
    uint32_t wtot = 0;
#pragma unroll
    for (int r = 0; r < kChainChunks; ++r) {
        const bool ok = cnt[r] > 0u;
        bal[r] = __ballot_sync(0xffffffffu, ok);
        wtot += __popc(bal[r]);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t d = ok ? (key[r] >> (8 * p)) & 255u : 0xffffffffu;
            const uint32_t peers = digit_peers(d, ok);
            if (ok && lane == __ffs(peers) - 1) atomicAdd(&s_h[p][d], (uint32_t)__popc(peers));
        }
    }
    if (lane == 0) s_warp[warp] = wtot;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = lane < kChainWarps ? s_warp[lane] : 0u;
        const uint32_t inc = warp_incl_scan(v);
        const uint32_t total = __shfl_sync(0xffffffffu, inc, kChainWarps - 1);
        const uint32_t excl = (uint32_t)chain_lookback(lb, tile, total, err, SG_LOOKBACK_COMPACT);
        if (lane < kChainWarps) s_warp[lane] = excl + inc - v;
        if (lane == 0 && tile == ntiles - 1) *d_nvalid = excl + total;
    }
    __syncthreads();
    uint32_t pos = s_warp[warp];
#pragma unroll
    for (int r = 0; r < kChainChunks; ++r) {
        if ((bal[r] >> lane) & 1u) {
            const uint32_t q = pos + __popc(bal[r] & ((1u << lane) - 1u));
            keys[q] = key[r];
            vals[q] = (uint32_t)(wbase + r * 32 + lane);
        }
        pos += __popc(bal[r]);
    }
    for (int i = threadIdx.x; i < 4 * 256; i += kChainThreads) {
        const uint32_t c = (&s_h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

__global__ void __launch_bounds__(kChainThreads)
k_pair_offsets(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ count, int64_t n,
               const uint32_t *__restrict__ d_nvalid, uint32_t *__restrict__ offsets,
               uint32_t *__restrict__ d_total, unsigned long long *__restrict__ lb,
               uint32_t *__restrict__ ticket, uint32_t *__restrict__ err)
{
    __shared__ uint32_t s_warp[kChainWarps];
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t nv = *d_nvalid;
    const int64_t ntiles = (nv + kChainTile - 1) / kChainTile;
    if (nv == 0) {
        if (tile == 0 && threadIdx.x == 0) *d_total = 0u;
        return;
    }
    if (tile >= ntiles) return;   // so is every later tile: nobody waits for this one
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wbase = tile * kChainTile + (int64_t)warp * 32 * kChainChunks;
    uint32_t c[kChainChunks];
#pragma unroll
    for (int r = 0; r < kChainChunks; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        c[r] = i < nv ? ids[i] : 0xffffffffu;
    }
    // an id is outside 0..n-1 only after a look-back wait of the depth sort
    // gave up (err set, the sort's output partly unwritten): count it as 0
#pragma unroll
    for (int r = 0; r < kChainChunks; ++r) c[r] = (int64_t)c[r] < n ? count[c[r]] : 0u;
    uint32_t run = 0;   // the warp's entries before chunk r
#pragma unroll
    for (int r = 0; r < kChainChunks; ++r) {
        const uint32_t inc = warp_incl_scan(c[r]);
        const uint32_t v = c[r];
        c[r] = run + inc - v;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) s_warp[warp] = run;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = lane < kChainWarps ? s_warp[lane] : 0u;
        const uint32_t inc = warp_incl_scan(v);
        const uint32_t total = __shfl_sync(0xffffffffu, inc, kChainWarps - 1);
        const unsigned long long excl = chain_lookback(lb, tile, total, err, SG_LOOKBACK_OFFSETS);
        if (lane < kChainWarps) s_warp[lane] = (uint32_t)excl + inc - v;
        if (lane == 0 && tile == ntiles - 1) {
            // saturated, so that a total of 2^32 pairs or more reads as an overflow
            const unsigned long long tot = excl + total;
            *d_total = tot > 0xffffffffull ? 0xffffffffu : (uint32_t)tot;
        }
    }
    __syncthreads();
    const uint32_t pre = s_warp[warp];
#pragma unroll
    for (int r = 0; r < kChainChunks; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        if (i < nv) offsets[i] = pre + c[r];
    }
}

sg_status depth_stage(const uint32_t *d_count, const float *d_depth, int64_t n, uint32_t *keys[2],
                      uint32_t *vals[2], uint32_t *d_scal, uint32_t *d_offsets, Frame &fr,
                      cudaStream_t st, int *result_buf)
{
    *result_buf = 0;
    if (n <= 0) {   // no projection kernel ran: clear the status word too
        SG_CUDA(cudaMemsetAsync(d_scal, 0, 4 * (kScalStatus + 1), st));
        return SG_OK;
    }
    if (n > (int64_t)kLbCount) {
        set_error("depth sort of %lld Gaussians exceeds 2^30", (long long)n);
        return SG_ERR_OVERFLOW;
    }
    // after the radix scratch, zeroed with it: two tickets, then one 64-bit
    // word per tile for each of the two chained scans
    const int64_t ntiles = (n + kChainTile - 1) / kChainTile;
    uint32_t *hist = nullptr;
    sg_status s =
        radix_prepare(n, 4, fr, st, &hist, depth_stage_words(n) - radix_scratch_words(n, 4));
    if (s != SG_OK) return s;
    static_assert(radix_scratch_words(1, 4) % 2 == 0, "64-bit chain words stay aligned");
    unsigned long long *chain = (unsigned long long *)(hist + radix_scratch_words(n, 4));
    uint32_t *tickets = (uint32_t *)chain;                 // [0] compaction, [1] offsets
    uint32_t *err = (uint32_t *)fr.scalars.p + kScalStatus;
    k_compact_depth<<<(unsigned)ntiles, kChainThreads, 0, st>>>(
        d_count, d_depth, n, ntiles, keys[0], vals[0], d_scal, hist, chain + 2, tickets, err);
    SG_LAUNCHED();
    if ((s = radix_sort_pairs(keys, vals, n, d_scal, 0, 32, fr, st, result_buf,
                              SG_LOOKBACK_DEPTH_SORT)) != SG_OK)
        return s;
    k_pair_offsets<<<(unsigned)ntiles, kChainThreads, 0, st>>>(
        vals[*result_buf], d_count, n, d_scal, d_offsets, d_scal + 1, chain + 2 + ntiles,
        tickets + 1, err);
    SG_LAUNCHED();
    return SG_OK;
}

// ------------------------------------------------------------------ binning

// Expand each valid Gaussian (depth order) into its (tile, Gaussian) pairs:
// pair o of Gaussian g goes to position offsets[g] + o, tile rows outer and
// columns inner.  Pairs at positions >= cap are not written (capacity mode:
// the caller learns of them from the dropped-pairs count).
// Balanced by pairs: block b writes pairs [b C, (b + 1) C) of the
// depth-ordered expansion (C = kBinChunk; pair p belongs to the valid
// Gaussian k with offsets[k] <= p < offsets[k + 1]).  The block first finds
// the owner of its first pair by a cooperative search over the offsets
// (256 samples per round), loads the offsets and ids of the at most C + 1
// Gaussians its pairs can belong to, then every thread places its pairs
// (owner by binary search in shared memory, tile from the owner's range).
// A Gaussian that covers thousands of tiles is spread over many blocks.
constexpr int kBinThreads = 256;
constexpr int kBinPasses = 3;         // tile ids up to 24 bits when k_bin counts the digits
constexpr int kBinChunk = 1024;

__global__ void __launch_bounds__(kBinThreads)
k_bin(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offsets,
      const uint32_t *__restrict__ d_scal, const int4 *__restrict__ tiles, int ntx, int wrap_x,
      uint32_t cap, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
      uint32_t *__restrict__ hist, int end_bit, const uint32_t *__restrict__ err)
{
    __shared__ uint32_t s_off[kBinChunk + 1], s_id[kBinChunk + 1];
    __shared__ uint32_t s_h[kBinPasses][256];
    const int t = threadIdx.x;
    const int passes = (end_bit + 7) / 8;
    for (int i = t; i < kBinPasses * 256; i += kBinThreads) (&s_h[0][0])[i] = 0u;
    const int64_t nvalid = d_scal[0];
    const int64_t K = min((int64_t)d_scal[1], (int64_t)cap);
    const int64_t p0 = (int64_t)blockIdx.x * kBinChunk;
    // after a look-back wait of the depth stage gave up, the ids and offsets
    // are not trustworthy (offsets may decrease): write nothing
    if (p0 >= K || nvalid == 0 || *err) return;
    const int64_t p1 = min(K, p0 + kBinChunk);
    // the owner of p0: the largest k with offsets[k] <= p0 (offsets[0] = 0,
    // strictly increasing: every valid Gaussian has a pair)
    int64_t lo = 0, hi = nvalid;
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + kBinThreads - 1) / kBinThreads;
        const int64_t idx = lo + t * step;
        const bool le = idx < hi && (int64_t)offsets[idx] <= p0;
        const int c = __syncthreads_count(le);
        lo = lo + (int64_t)(c - 1) * step;
        hi = min(hi, lo + step);
    }
    const int64_t k0 = lo;
    const int nk = (int)min((int64_t)kBinChunk + 1, nvalid - k0);
    for (int i = t; i < nk; i += kBinThreads) {
        s_off[i] = offsets[k0 + i];
        s_id[i] = ids[k0 + i];
    }
    __syncthreads();
    for (int r0 = 0; r0 < kBinChunk; r0 += kBinThreads) {
        const int64_t pos = p0 + r0 + t;
        const bool in = pos < p1;
        uint32_t key = 0u;
        if (in) {
            int a = 0, b = nk;             // the last j with s_off[j] <= pos
            while (b - a > 1) {
                const int m = (a + b) >> 1;
                if ((int64_t)s_off[m] <= pos) a = m; else b = m;
            }
            const uint32_t g = s_id[a];
            const int4 r = tiles[g];
            const uint32_t local = (uint32_t)(pos - s_off[a]), w = (uint32_t)(r.y - r.x + 1);
            const int ty = min(r.w, r.z + (int)(local / w));   // within the range, always
            int x = r.x + (int)(local % w);
            if (wrap_x) { x %= ntx; if (x < 0) x += ntx; }
            key = (uint32_t)(ty * ntx + x);
            keys[pos] = key;
            vals[pos] = g;
        }
        if (hist) {
            // the digit counts of every tile-sort pass
            for (int p = 0; p < passes; ++p) {
                const int bits = end_bit - 8 * p < 8 ? end_bit - 8 * p : 8;
                const uint32_t dg = (key >> (8 * p)) & ((1u << bits) - 1u);
                const uint32_t peers = digit_peers(dg, in);
                if (in && (t & 31) == __ffs(peers) - 1) atomicAdd(&s_h[p][dg], (uint32_t)__popc(peers));
            }
        }
    }
    if (hist) {
        __syncthreads();
        for (int i = t; i < passes * 256; i += kBinThreads) {
            const uint32_t c = (&s_h[0][0])[i];
            if (c) atomicAdd(&hist[i], c);
        }
    }
}

sg_status bin_pairs(const uint32_t *d_ids, const uint32_t *d_offsets, const uint32_t *d_nvalid,
                    const int4 *d_tiles, int ntx, int wrap_x, int64_t cap, uint32_t *d_keys,
                    uint32_t *d_vals, cudaStream_t st, const uint32_t *d_err, uint32_t *d_hist,
                    int end_bit)
{
    if (cap <= 0) return SG_OK;
    if (d_hist && (end_bit < 1 || end_bit > 8 * kBinPasses)) {
        set_error("internal: %d-bit tile ids", end_bit);
        return SG_ERR_INVALID;
    }
    k_bin<<<(unsigned)((cap + kBinChunk - 1) / kBinChunk), kBinThreads, 0, st>>>(
        d_ids, d_offsets, d_nvalid, d_tiles, ntx, wrap_x, (uint32_t)cap, d_keys, d_vals, d_hist,
        end_bit, d_err);
    SG_LAUNCHED();
    return SG_OK;
}

// Per-tile [start, end) of the sorted pairs, and for camera lists (kMask)
// a per-pair 32-bit word of the tile's pixel columns (bits 0-15) and rows
// (bits 16-31) whose centres lie inside the Gaussian's extent box, by the
// same float comparisons as the per-ray test.  A compositing warp gets from
// it, in a few integer operations, whether the entry reaches its 8x4
// sub-block and which of its lanes the box holds, so it never stages an
// entry that no live ray of its sub-block can see and loads no box.  After a
// look-back wait gave up (*err) the pairs may hold stale tile ids: every
// range stays empty (zeroed before the launch).
// Each thread takes kRangePer consecutive pairs, their loads (keys, ids,
// then the boxes by id) issued together, so that a thread waits for two
// rounds of loads for all of them.
constexpr int kRangePer = 4;

template <bool kMask>
__global__ void __launch_bounds__(256)
k_ranges(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ d_K,
         uint2 *__restrict__ ranges, const uint32_t *__restrict__ ids,
         const float4 *__restrict__ rects, int ntx, uint32_t *__restrict__ mask,
         const uint32_t *__restrict__ err)
{
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kRangePer;
    const int64_t K = *d_K;
    if (i0 >= K || *err) return;
    uint32_t t[kRangePer], id[kRangePer];
    float4 rc[kRangePer];
#pragma unroll
    for (int j = 0; j < kRangePer; ++j) {
        const bool in = i0 + j < K;
        t[j] = in ? keys[i0 + j] : 0u;
        if (kMask) id[j] = in ? ids[i0 + j] : 0u;
    }
    const uint32_t before = i0 > 0 ? keys[i0 - 1] : 0u;
    const uint32_t after = i0 + kRangePer < K ? keys[i0 + kRangePer] : 0u;
    if (kMask) {
#pragma unroll
        for (int j = 0; j < kRangePer; ++j)
            if (i0 + j < K) rc[j] = rects[id[j]];   // the extent box, 16 B per Gaussian
    }
#pragma unroll
    for (int j = 0; j < kRangePer; ++j) {
        const int64_t i = i0 + j;
        if (i >= K) break;
        const uint32_t left = j > 0 ? t[j - 1] : before;
        const uint32_t right = j + 1 < kRangePer ? t[j + 1] : after;
        if (i == 0 || left != t[j]) ranges[t[j]].x = (uint32_t)i;
        if (i == K - 1 || right != t[j]) ranges[t[j]].y = (uint32_t)(i + 1);
        if (kMask) {
            const int tx = (int)(t[j] % (uint32_t)ntx), ty = (int)(t[j] / (uint32_t)ntx);
            uint32_t cols = 0, rows = 0;
#pragma unroll
            for (int c = 0; c < kTile; ++c) {
                const float x = (float)(tx * kTile + c) + 0.5f;
                const float y = (float)(ty * kTile + c) + 0.5f;
                cols |= (uint32_t)(x >= rc[j].x && x <= rc[j].y) << c;
                rows |= (uint32_t)(y >= rc[j].z && y <= rc[j].w) << c;
            }
            mask[i] = cols | (rows << 16);
        }
    }
}

sg_status tile_ranges(const uint32_t *d_keys, const uint32_t *d_K, int64_t K_max, uint2 *d_ranges,
                      int64_t ntiles, cudaStream_t st, const uint32_t *d_err,
                      const uint32_t *d_ids, const float4 *d_rects, int ntx, uint32_t *d_words)
{
    SG_CUDA(cudaMemsetAsync(d_ranges, 0, sizeof(uint2) * ntiles, st));
    if (K_max == 0) return SG_OK;
    const unsigned grid = (unsigned)((K_max + 256 * kRangePer - 1) / (256 * kRangePer));
    if (d_words)
        k_ranges<true><<<grid, 256, 0, st>>>(d_keys, d_K, d_ranges, d_ids, d_rects, ntx, d_words,
                                             d_err);
    else
        k_ranges<false><<<grid, 256, 0, st>>>(d_keys, d_K, d_ranges, nullptr, nullptr, 0, nullptr,
                                              d_err);
    SG_LAUNCHED();
    return SG_OK;
}

// LiDAR lists: per-tile ranges, and per pair the ray masks of the work
// items of its tile (k-th item of the tile: lmask[k * K_max + i]), so that
// the compositing walks skip entries that reach none of their rays without
// loading their records.  A ray is in the box iff its column's azimuth (the
// alias nearest the box centre) and its beam's elevation are, so the mask
// takes one test per column and one per beam of the item.  Both the forward
// and the backward walks read these masks, so they take the same decisions.
__global__ void k_ranges_lidar(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ d_K,
                               int64_t K_max, uint2 *__restrict__ ranges,
                               const uint32_t *__restrict__ ids, const float4 *__restrict__ rects,
                               const uint2 *__restrict__ tile_items,
                               const LidarItemRays *__restrict__ tab,
                               uint32_t *__restrict__ lmask, const uint32_t *__restrict__ err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t K = *d_K;
    if (i >= K || *err) return;
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == K - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
    const float4 rc = rects[ids[i]];
    const float cx = 0.5f * (rc.x + rc.y);
    const uint2 ti = tile_items[t];
    for (uint32_t k = 0; k < ti.y; ++k) {
        const LidarItemRays &R = tab[ti.x + k];
        uint32_t mc = 0u, me = 0u;
        for (int s = 0; s < R.ncols; ++s) {
            const float az = R.col_az[s];
            const float ra = az + 360.f * rintf((cx - az) * (1.f / 360.f));
            mc |= (ra >= rc.x && ra <= rc.y) ? R.col_bits[s] : 0u;
        }
        for (int j = 0; j < R.nbeams; ++j) {
            const float el = R.beam_el[j];
            me |= (el >= rc.z && el <= rc.w) ? R.beam_bits[j] : 0u;
        }
        lmask[(int64_t)k * K_max + i] = mc & me;
    }
}

sg_status lidar_tile_ranges(const uint32_t *d_keys, const uint32_t *d_K, int64_t K_max,
                            uint2 *d_ranges, int64_t ntiles, cudaStream_t st,
                            const uint32_t *d_err, const uint32_t *d_ids,
                            const float4 *d_rects, const Lidar &L, uint32_t *d_lmask)
{
    SG_CUDA(cudaMemsetAsync(d_ranges, 0, sizeof(uint2) * ntiles, st));
    if (K_max == 0) return SG_OK;
    k_ranges_lidar<<<(unsigned)((K_max + 255) / 256), 256, 0, st>>>(
        d_keys, d_K, K_max, d_ranges, d_ids, d_rects, L.d_tile_items, L.d_item_ray_tab, d_lmask,
        d_err);
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

extern "C" sg_status sg_debug_lookback(uint32_t max_spins, int hold_site, int64_t hold_tile)
{
    if (hold_site < 0 || hold_site > SG_LOOKBACK_TILE_SORT || hold_tile < -1) {
        sg::set_error("sg_debug_lookback: site %d / tile %lld out of range", hold_site,
                      (long long)hold_tile);
        return SG_ERR_INVALID;
    }
    const uint32_t spins = max_spins ? max_spins : sg::kLbSpinsDefault;
    const long long tile = hold_site ? (long long)hold_tile : -1;
    SG_CUDA(cudaDeviceSynchronize());   // no kernel reads them meanwhile
    SG_CUDA(cudaMemcpyToSymbol(sg::g_lb_spins, &spins, sizeof(spins)));
    SG_CUDA(cudaMemcpyToSymbol(sg::g_hold_site, &hold_site, sizeof(hold_site)));
    SG_CUDA(cudaMemcpyToSymbol(sg::g_hold_tile, &tile, sizeof(tile)));
    return SG_OK;
}
