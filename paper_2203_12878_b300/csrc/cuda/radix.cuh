// One pass of the stable LSD radix sort (onesweep form): every block ranks a
// tile of keys by one 8-bit digit, learns where earlier tiles put the same
// digits through a decoupled look-back over per-tile, per-digit status words
// (every wait bounded), and scatters the tile through shared memory so that
// each digit's run leaves the block as consecutive stores.
//
// Digit bases come from the pass's global digit histogram, built upstream.
// Status word: flag (bits 62..63: 1 tile aggregate, 2 inclusive prefix),
// launch tag (bits 40..61, so words of earlier launches are ignored), count
// (bits 0..39).
#pragma once

#include <cstdint>

namespace drf {
namespace radix {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 40) - 1;
constexpr int kTagShift = 40;
constexpr unsigned long long kTagMask = (1ull << 22) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;   // ~ a second of waiting at most
constexpr int kBins = 256;
constexpr long long kNoWrite = -(1ll << 62);  // marks a digit whose run would leave the output

struct PassArgs {
    const unsigned long long *src;
    unsigned long long *dst;
    uint64_t n;
    uint32_t shift;                  // first bit of the digit
    uint32_t nbits;                  // digit width (<= 8)
    const unsigned long long *hist;  // [256] global digit counts of this pass
    unsigned long long *status;      // [tiles][256] look-back words
    unsigned long long *tile_counter;
    unsigned long long tag;          // launch tag, already shifted into place
    unsigned int *flags;             // bit 1: look-back timeout, bit 2: out-of-range scatter
    uint32_t spin_limit;             // look-back waits per digit before giving up (kSpinLimit normally)
    // test hook: tile 0 publishes no status, so that the waits of the tiles
    // after it run out (and the pass reports a look-back timeout)
    uint32_t stall_first;
};

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ void st_volatile(unsigned long long *p, unsigned long long v)
{
    *reinterpret_cast<volatile unsigned long long *>(p) = v;
}

template <int BLOCK, int ITEMS>
struct PassShared {
    static constexpr int kWarps = BLOCK / 32;
    static constexpr int kTile = BLOCK * ITEMS;
    unsigned long long keys[kTile];
    uint32_t whist[kWarps][kBins];        // per-warp digit counts, then per-warp scatter bases
    long long gdelta[kBins];              // global position minus tile position, per digit
    unsigned long long scan[kWarps];
    uint32_t tile;
};

// The pass body; BLOCK threads, BLOCK >= 256 (one thread per digit for the
// digit-wise steps).
// Digit of a key at bit `shift` (uniform over the launch): one funnel shift
// of the key's two 32-bit halves.
__device__ __forceinline__ uint32_t digit_of(unsigned long long k, uint32_t shift, uint32_t mask)
{
    const uint32_t lo = (uint32_t)k, hi = (uint32_t)(k >> 32);
    const uint32_t v = shift < 32 ? __funnelshift_r(lo, hi, shift) : hi >> (shift - 32);
    return v & mask;
}

template <int BLOCK, int ITEMS, int WINDOW = 4>
__device__ __forceinline__ void pass(const PassArgs &A, PassShared<BLOCK, ITEMS> &sh)
{
    static_assert(BLOCK >= kBins && BLOCK % 32 == 0, "one thread per digit");
    constexpr int kLookWindow = WINDOW;   // predecessor statuses read per look-back step
    constexpr int kWarps = BLOCK / 32;
    constexpr int kTile = BLOCK * ITEMS;
    constexpr int kWarpKeys = 32 * ITEMS;
    const uint32_t t = threadIdx.x, lane = t & 31, wid = t / 32;
    const uint32_t dmask = (1u << A.nbits) - 1;
    const uint32_t shift = A.shift;

    for (int i = t; i < kWarps * kBins; i += BLOCK) (&sh.whist[0][0])[i] = 0;
    if (t == 0) sh.tile = (uint32_t)atomicAdd(A.tile_counter, 1ull);
    // global start of every digit: exclusive scan of the pass histogram
    unsigned long long h = t < kBins ? A.hist[t] : 0, incl = h;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh.scan[wid] = incl;
    __syncthreads();
    unsigned long long dbase = incl - h;
    for (uint32_t i = 0; i < wid; i++) dbase += sh.scan[i];
    const uint32_t tile = sh.tile;
    const uint64_t base = (uint64_t)tile * kTile;
    const uint64_t n = A.n;
    const uint32_t valid_n = (uint32_t)min((uint64_t)kTile, n - base);
    const unsigned long long *src = A.src + base;

    // load: warp w owns keys [w*32*ITEMS, (w+1)*32*ITEMS) of the tile, 32
    // consecutive keys per round, so that (round, lane) order is memory order
    unsigned long long key[ITEMS];
    const uint32_t wofs = wid * kWarpKeys + lane;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        const uint32_t idx = wofs + i * 32;
        key[i] = idx < valid_n ? src[idx] : 0;
    }
    // rank inside the warp, stable in memory order: lanes with equal digits
    // meet in one match; the lowest of them claims the run in the warp's
    // counter and hands the old count to the others
    uint32_t rank[ITEMS];
    uint32_t digs[(ITEMS + 3) / 4];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        const bool valid = wofs + i * 32 < valid_n;
        const uint32_t d = digit_of(key[i], shift, dmask);
        if (i % 4 == 0) digs[i / 4] = 0;
        digs[i / 4] |= d << (8 * (i % 4));
        const unsigned peers = __match_any_sync(kFull, valid ? d : 0x100u + lane);
        const uint32_t below = __popc(peers & lt);
        uint32_t prior = 0;
        if (valid && below == 0) prior = atomicAdd(&sh.whist[wid][d], (uint32_t)__popc(peers));
        prior = __shfl_sync(kFull, prior, __ffs(peers) - 1);
        rank[i] = prior + below;
    }
    __syncthreads();
    // per digit: exclusive offsets of the warps, and the tile's count
    uint32_t cnt = 0;
    if (t < kBins) {
        for (int w = 0; w < kWarps; w++) {
            uint32_t c = sh.whist[w][t];
            sh.whist[w][t] = cnt;
            cnt += c;
        }
    }
    // publish the tile aggregate for digit t, then look back
    unsigned long long excl = 0;
    if (t < kBins) {
        unsigned long long *my = A.status + (uint64_t)tile * kBins + t;
        if (!(A.stall_first && tile == 0)) st_volatile(my, (tile == 0 ? kFlagPrefix : kFlagAgg) | A.tag | cnt);
        if (tile > 0) {
            int64_t j = (int64_t)tile - 1;
            uint32_t spins = 0;
            bool gave_up = false;
            while (j >= 0) {
                unsigned long long w[kLookWindow];
#pragma unroll
                for (int u = 0; u < kLookWindow; u++)
                    w[u] = j - u >= 0 ? ld_volatile(A.status + (uint64_t)(j - u) * kBins + t) : (kFlagPrefix | A.tag);
                int used = 0;
                bool stop = false, wait = false;
#pragma unroll
                for (int u = 0; u < kLookWindow; u++) {
                    if (stop || wait) continue;
                    const unsigned long long s = w[u];
                    if ((s & (kTagMask << kTagShift)) != A.tag || (s >> 62) == 0) { wait = true; continue; }
                    excl += s & kValueMask;
                    used++;
                    if ((s >> 62) == 2) stop = true;
                }
                if (stop) break;
                j -= used;
                if (wait) {
                    if (++spins > A.spin_limit) { gave_up = true; break; }
                    __nanosleep(spins < 64 ? 32 : 256);
                }
            }
            if (gave_up) atomicOr(A.flags, 1u);
            st_volatile(my, kFlagPrefix | A.tag | ((excl + cnt) & kValueMask));
        }
    }
    // tile-local start of every digit (block scan of the counts)
    uint32_t tincl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, tincl, o);
        if (lane >= o) tincl += y;
    }
    __syncthreads();
    if (lane == 31) sh.scan[wid] = tincl;
    __syncthreads();
    uint32_t tstart = tincl - cnt;
    for (uint32_t i = 0; i < wid; i++) tstart += (uint32_t)sh.scan[i];
    if (t < kBins) {
        // this tile's run of digit t goes to [dbase + excl, + cnt): check it
        // lies inside the output once per digit instead of once per key
        const unsigned long long start = dbase + excl;
        const bool inside = start + cnt <= n;
        if (!inside && cnt) atomicOr(A.flags, 2u);   // histogram and keys disagree
        sh.gdelta[t] = inside ? (long long)start - (long long)tstart : kNoWrite;
        for (int w = 0; w < kWarps; w++) sh.whist[w][t] += tstart;   // scatter base of (warp, digit)
    }
    __syncthreads();
    // scatter into tile order in shared memory, then stream each digit's run out
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
        if (wofs + i * 32 < valid_n) {
            const uint32_t d = (digs[i / 4] >> (8 * (i % 4))) & 0xFF;
            sh.keys[sh.whist[wid][d] + rank[i]] = key[i];
        }
    }
    __syncthreads();
    for (uint32_t j = t; j < valid_n; j += BLOCK) {
        const unsigned long long k = sh.keys[j];
        const long long g = sh.gdelta[digit_of(k, shift, dmask)];
        if (g != kNoWrite) A.dst[g + (long long)j] = k;
    }
}

}  // namespace radix
}  // namespace drf
