// K2 counts, K3 coarse entries, K4 radix sort, K5 tile lists and ranges.
//
// The pair lists carry the canonical index of each Gaussian: this is the permutation pi of Eq. 10
// ("a GPU sort yields a permutation mapping sorted index i to canonical index pi(i)").  Parameters
// are never reordered; the compositing kernels gather by pi and the backward scatters gradients to
// pi (index-mapped gradient scattering).
//
// Every tile's list holds the Gaussians that reach it in depth order, ties in canonical order: the
// order of the stable sort of (tile << 32 | depth bits) pairs.  It is built in two levels.  The
// Gaussians are sorted by depth (32-bit keys, ties kept in canonical order); each then emits one
// coarse entry per super-tile (kSuperW x kSuperH tiles) its tile rectangle overlaps, in depth
// order; a stable radix sort by super-tile id groups the entries by super-tile, still in depth
// order inside each group.  The fine stage gives each entry a 32-bit mask of the super-tile's tiles
// the Gaussian reaches (the projection's reach test), counts each tile's entries per block of
// kFineBlock (a warp's 32 masks transposed in five shuffle stages, so lane x holds the lanes that
// reach tile x), scans those counts, and writes each entry's canonical index at its tile's first
// pair + the entries of the tile before it.  The pair buffer is laid out
// super-tile by super-tile, tiles row-major inside; a tile's list is [ranges[t].x, ranges[t].y).
// The pair count is the sum of the projection's reached-tile counts, known before any list is
// built; pairs beyond the capacity are not written (the status word records the overflow and the
// capacity needed), so no host synchronisation sits between projection and compositing.
//
// The radix sort is least-significant-digit first, 8-bit digits, over the bits that can be
// non-zero (32 depth bits for the Gaussians, ceil(log2 super-tiles) bits for the coarse entries;
// the caller's low key bits of the 64-bit keys of the allocation-free entry point); the last digit
// is masked to what is left of the bit range.  The digit totals of every pass come from one
// up-front histogram; each pass is then one launch that ranks a tile's keys with warp ballots and
// finds the tile's place by decoupled look-back over the tiles before it (bounded waits, see
// k_onesweep).
//
// The kernels of a render's binning start with pdl_begin() and are launched by launch_pdl (the
// timeout self-test launches plainly): the next one is scheduled while the current one's last
// CTAs run and waits for them before it touches memory.
// The scratch these kernels expect zeroed (look-back words, digit totals, counters, ranges) is
// cleared by the projection before them (render_zero_plan), or by memsets when the caller says so.
#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
static_assert(kSortThreads == kRadix, "one thread per digit in the sort kernels");

// ---------------------------------------------------------------------------------------------
// K2: pair count and coarse entry counts
// ---------------------------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

// super-tile rectangle [sx0, sx1) x [sy0, sy1) of a tile rectangle (x0 | y0 << 16, x1 | y1 << 16)
__device__ __forceinline__ void super_rect(uint2 r, uint32_t& sx0, uint32_t& sy0, uint32_t& sx1, uint32_t& sy1) {
    sx0 = (r.x & 0xffffu) / kSuperW;
    sy0 = (r.x >> 16) / kSuperH;
    sx1 = ((r.y & 0xffffu) + kSuperW - 1) / kSuperW;
    sy1 = ((r.y >> 16) + kSuperH - 1) / kSuperH;
}

// Exclusive scan of `count` values by one CTA (a whole number of warps, at most 1024 threads),
// kV consecutive values per thread and step: load(i) gives value i, store(i, prefix) receives its
// exclusive prefix; returns the total to every thread.  Every thread of the CTA calls it.
template <class Load, class Store>
__device__ unsigned long long cta_scan(int count, Load load, Store store) {
    constexpr int kV = 8;
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < count; base += blockDim.x * kV) {
        const int first = base + threadIdx.x * kV;
        unsigned long long v[kV], tsum = 0;
#pragma unroll
        for (int k = 0; k < kV; ++k) {
            v[k] = first + k < count ? load(first + k) : 0ull;
            tsum += v[k];
        }
        unsigned long long incl = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long w = lane < nw ? s_warp[lane] : 0ull;
            unsigned long long wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long t = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi += t;
            }
            if (lane < nw) s_warp[lane] = wi - w;
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        unsigned long long run = carry + s_warp[warp] + incl - tsum;
#pragma unroll
        for (int k = 0; k < kV; ++k) {
            if (first + k < count) store(first + k, run);
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = run;
        __syncthreads();
    }
    return s_carry;
}

// Is this CTA the last of the grid to get here?  Each CTA's writes before the call are visible to
// the last one (fence before the ticket, fence after); the last CTA resets the ticket.  No CTA
// waits for another.
__device__ __forceinline__ bool last_cta(uint32_t* ticket) {
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (s_last) *ticket = 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// Per block of kProjBlock depth-ordered Gaussians (the coarse emission's CTAs): coarse entries
// (super-tiles of the rectangle) into block_sums; reached tiles added into pair_count (zeroed
// before).  A CTA takes kCountItems such blocks, one Gaussian of each per thread, so each thread
// has that many independent gathers in flight.  The last CTA then scans the per-block counts into
// their offsets and sets the coarse total, the coarse sort's CTA count, the capacity the render
// needs (pairs, and the coarse stage's entries and counters) and the capacity check.
constexpr int kCountItems = 4;
__global__ void __launch_bounds__(kProjBlock)
k_coarse_counts(int64_t n, int64_t capacity, int64_t supers, const uint32_t* __restrict__ perm, Scratch sc) {
    pdl_begin();
    const int64_t nbk = (n + kProjBlock - 1) / kProjBlock;  // blocks of the emission
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t g[kCountItems], reached[kCountItems], area[kCountItems];
    uint2 rect[kCountItems];
#pragma unroll
    for (int k = 0; k < kCountItems; ++k) {
        const int64_t i = ((int64_t)blockIdx.x * kCountItems + k) * kProjBlock + threadIdx.x;
        g[k] = i < n ? perm[i] : 0xffffffffu;
    }
#pragma unroll
    for (int k = 0; k < kCountItems; ++k) {
        const bool valid = g[k] != 0xffffffffu;
        reached[k] = valid ? sc.touched[g[k]] : 0u;
        rect[k] = valid ? sc.rect[g[k]] : make_uint2(0u, 0u);
    }
    __shared__ uint32_t s_a[kCountItems][kProjBlock / 32], s_r[kProjBlock / 32];
    uint32_t rsum = 0;
#pragma unroll
    for (int k = 0; k < kCountItems; ++k) {
        area[k] = 0;
        if (reached[k]) {
            uint32_t sx0, sy0, sx1, sy1;
            super_rect(rect[k], sx0, sy0, sx1, sy1);
            area[k] = (sx1 - sx0) * (sy1 - sy0);
        }
        const uint32_t wa = __reduce_add_sync(kFull, area[k]);
        if (lane == 0) s_a[k][warp] = wa;
        rsum += reached[k];
    }
    const uint32_t wr = __reduce_add_sync(kFull, rsum);
    if (lane == 0) s_r[warp] = wr;
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool in = threadIdx.x < kProjBlock / 32;
#pragma unroll
        for (int k = 0; k < kCountItems; ++k) {
            const uint32_t a = __reduce_add_sync(kFull, in ? s_a[k][threadIdx.x] : 0u);
            const int64_t b = (int64_t)blockIdx.x * kCountItems + k;
            if (threadIdx.x == 0 && b < nbk) sc.block_sums[b] = a;
        }
        const unsigned long long r = __reduce_add_sync(kFull, in ? s_r[threadIdx.x] : 0u);
        if (threadIdx.x == 0 && r) atomicAdd(sc.pair_count, r);
    }
    if (!last_cta(&sc.bin_ticket[0])) return;
    const unsigned long long Ce = cta_scan(
        (int)nbk, [&](int k) { return (unsigned long long)__ldcg(&sc.block_sums[k]); },
        [&](int k, unsigned long long v) { sc.block_offsets[k] = v; });
    if (threadIdx.x == 0) {
        const unsigned long long P = atomicAdd(sc.pair_count, 0ull);
        *sc.coarse_count = Ce;
        const unsigned long long kept = Ce < (unsigned long long)capacity ? Ce : (unsigned long long)capacity;
        *sc.sort_blocks = (uint32_t)((kept + kSortTile - 1) / kSortTile);
        const unsigned long long c = coarse_need(Ce, (unsigned long long)supers);
        const unsigned long long need = P > c ? P : c;
        *sc.pair_need = need;
        if (need > (unsigned long long)capacity) atomicOr(sc.status, kStatusCapacity);
    }
}

// Transpose of the warp's 32 x 32 bit matrix (lane l holds row l): lane x returns column x, whose
// bit l is bit x of lane l's word.  Five stages; at stage j the lanes l and l ^ j swap the block of
// bits b with b & j set (upper lane l) against the block with b & j clear (lower lane l ^ j).
__device__ __forceinline__ uint32_t warp_transpose(uint32_t x, int lane) {
    constexpr uint32_t kMask[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int j = 16 >> k;
        const uint32_t m = kMask[k];
        const uint32_t o = __shfl_xor_sync(kFull, x, j);
        x = (lane & j) ? ((x & ~m) | ((o & ~m) >> j)) : ((x & m) | ((o & m) << j));
    }
    return x;
}

// Reach mask of one entry per lane (warp-collective): tiles of the super-tile at tile (bx, by) (each
// lane its own) that Gaussian g reaches, bit (ty - by) kSuperW + tx - bx.  Rectangles of <= 32 tiles: read row by row
// from the projection's reach mask.  Larger ones: the warp runs the projection's reach test over
// all such lanes' candidate tiles together, 32 per round (candidate k by lane k mod 32, its lane
// found by a shuffle binary search over the lanes' inclusive candidate counts), so one large
// Gaussian does not hold its warp for 32 tests.
__device__ __forceinline__ uint32_t entry_mask(bool valid, uint32_t g, uint2 r, uint32_t hm, uint32_t bx, uint32_t by,
                                               int T, const Scratch& sc, int lane, uint32_t* s_big) {
    uint32_t mask = 0, ncand = 0, X0 = 0, Y0 = 0, wX = 1;
    float u = 0.f, v = 0.f, ca = 0.f, cb = 0.f, cc = 0.f, ssx = 0.f, ssy = 0.f;
    if (valid) {
        const uint32_t x0 = r.x & 0xffffu, y0 = r.x >> 16, x1 = r.y & 0xffffu, y1 = r.y >> 16;
        X0 = max(x0, bx);
        Y0 = max(y0, by);
        const uint32_t X1 = min(x1, bx + kSuperW), Y1 = min(y1, by + kSuperH);
        const uint32_t w = x1 - x0;
        wX = X1 - X0;  // >= 1: the super-tile lies in the Gaussian's super-tile rectangle
        if (w * (y1 - y0) <= 32u) {
            const uint32_t row = (1u << wX) - 1u;
            for (uint32_t ty = Y0; ty < Y1; ++ty)
                mask |= ((hm >> ((ty - y0) * w + (X0 - x0))) & row) << ((ty - by) * kSuperW + (X0 - bx));
        } else {
            ncand = wX * (Y1 - Y0);
            const float4 p = sc.xyo[g], q = sc.conic[g];
            u = p.x;
            v = p.y;
            ca = q.x;
            cb = q.y;
            cc = q.z;
            ssx = __fdiv_rn(q.y, q.x);
            ssy = __fdiv_rn(q.y, q.z);
        }
    }
    uint32_t incl = ncand;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31), first = incl - ncand;
    if (total) {  // warp-uniform
        s_big[lane] = 0u;
        __syncwarp();
        for (uint32_t b = 0; b < total; b += 32) {
            const uint32_t k = b + (uint32_t)lane;
            int lo = 0, hi = 31;  // owner of candidate k: the first lane whose inclusive count exceeds k
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                const int mid = (lo + hi) >> 1;
                const uint32_t im = __shfl_sync(kFull, incl, mid);
                if (lo < hi) {
                    if (im > k) hi = mid;
                    else lo = mid + 1;
                }
            }
            const uint32_t of = __shfl_sync(kFull, first, lo), ow = __shfl_sync(kFull, wX, lo);
            const uint32_t ox = __shfl_sync(kFull, X0, lo), oy = __shfl_sync(kFull, Y0, lo);
            const float ou = __shfl_sync(kFull, u, lo), ov = __shfl_sync(kFull, v, lo);
            const float oa = __shfl_sync(kFull, ca, lo), ob = __shfl_sync(kFull, cb, lo), oc = __shfl_sync(kFull, cc, lo);
            const float osx = __shfl_sync(kFull, ssx, lo), osy = __shfl_sync(kFull, ssy, lo);
            const uint32_t obx = __shfl_sync(kFull, bx, lo), oby = __shfl_sync(kFull, by, lo);  // owner's super-tile
            if (k < total) {
                const uint32_t local = k - of, dy = local / ow, dx = local - dy * ow;
                const uint32_t tx = ox + dx, ty = oy + dy;
                if (tile_hit(ou, ov, oa, ob, oc, osx, osy, (int)tx, (int)ty, T))
                    atomicOr(&s_big[lo], 1u << ((ty - oby) * kSuperW + (tx - obx)));
            }
        }
        __syncwarp();
        mask |= s_big[lane];
        __syncwarp();
    }
    return mask;
}

// ---------------------------------------------------------------------------------------------
// K3: coarse entries of one CTA's Gaussians in depth order, super-tiles row-major inside each
// Gaussian's super-tile rectangle: key = super-tile id, value = the entry's own position e0, and at
// e0 the Gaussian's canonical index and its reach mask of the super-tile (rectangles of <= 32
// tiles: read from their reach bits; larger ones whose super-tile rectangle spans at most 2 x 2:
// the projection's masks; the rest: entry_mask).  Each warp walks
// the entries of its own 32 Gaussians, 32 per round (entry k by lane k mod 32; its Gaussian found
// by a shuffle binary search over the lanes' inclusive entry counts).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kProjBlock)
k_coarse_emit(int64_t n, int SX, int T, int64_t capacity, const uint32_t* __restrict__ perm, Scratch sc,
              uint32_t* __restrict__ gidx, uint32_t* __restrict__ gmask, int passes, uint32_t last_mask,
              const RenderDesc* __restrict__ renders, int R) {
    pdl_begin();
    __shared__ uint32_t s_sx0[kProjBlock], s_sy0[kProjBlock], s_sw[kProjBlock];
    __shared__ uint32_t s_SX[kProjBlock], s_base[kProjBlock], s_gid[kProjBlock], s_hm[kProjBlock];
    __shared__ uint2 s_rect[kProjBlock];
    __shared__ uint4 s_sm[kProjBlock];
    __shared__ uint32_t s_warp[kProjBlock / 32];
    __shared__ uint32_t s_big[kProjBlock / 32][32];
    __shared__ uint32_t s_hist[4][kRadix];  // digit counts of the written keys, pass by pass
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t i = (int64_t)blockIdx.x * kProjBlock + t;
    for (int k = t; k < 4 * kRadix; k += kProjBlock) (&s_hist[0][0])[k] = 0u;
    uint32_t cnt = 0;
    if (i < n) {
        const uint32_t g = perm[i];
        s_gid[t] = g;
        if (sc.touched[g]) {
            const uint2 r = sc.rect[g];
            uint32_t sx0, sy0, sx1, sy1;
            super_rect(r, sx0, sy0, sx1, sy1);
            s_sx0[t] = sx0;
            s_sy0[t] = sy0;
            s_sw[t] = sx1 - sx0;
            cnt = (sx1 - sx0) * (sy1 - sy0);
            s_rect[t] = r;
            const uint32_t area = ((r.y & 0xffffu) - (r.x & 0xffffu)) * ((r.y >> 16) - (r.x >> 16));
            s_hm[t] = area <= 32u ? sc.hitmask[g] : 0u;
            if (area <= 32u) s_sw[t] |= 0x40000000u;                          // masks from hitmask
            else if (sx1 - sx0 <= 2u && sy1 - sy0 <= 2u) s_sm[t] = sc.smask[g];  // projection's masks
            else s_sw[t] |= 0x80000000u;                                      // entry_mask
            s_SX[t] = (uint32_t)SX;
            s_base[t] = 0;
            if (renders) {  // batch: item g belongs to the last render whose first item is <= g
                int lo = 0, hi = R - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (renders[mid].item_base <= (int64_t)g) lo = mid;
                    else hi = mid - 1;
                }
                s_SX[t] = (uint32_t)renders[lo].SX;
                s_base[t] = (uint32_t)renders[lo].super_base;
            }
        }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t first = incl - cnt;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();  // also publishes the lanes' records in shared memory
    uint32_t before = 0;
#pragma unroll
    for (int w = 0; w < kProjBlock / 32; ++w) before += w < warp ? s_warp[w] : 0u;
    const unsigned long long out = sc.block_offsets[blockIdx.x] + before;
    uint32_t* ck = reinterpret_cast<uint32_t*>(sc.keys[0]);
    for (uint32_t b = 0; b < total; b += 32) {  // warp-uniform
        const uint32_t k = b + (uint32_t)lane;
        int lo = 0, hi = 31;  // owner of entry k: the first lane whose inclusive count exceeds k
#pragma unroll
        for (int step = 0; step < 5; ++step) {
            const int mid = (lo + hi) >> 1;
            const uint32_t im = __shfl_sync(kFull, incl, mid);
            if (lo < hi) {
                if (im > k) hi = mid;
                else lo = mid + 1;
            }
        }
        const uint32_t ofirst = __shfl_sync(kFull, first, lo);
        const bool valid = k < total;
        const int o = warp * 32 + lo;
        uint32_t sx = 0, sy = 0, slot = 0, g = 0, how = 0;
        uint2 r = make_uint2(0u, 0u);
        uint32_t hm = 0;
        if (valid) {
            const uint32_t local = k - ofirst, w = s_sw[o] & 0x3fffffffu;
            const uint32_t dy = local / w, dx = local - dy * w;
            sx = s_sx0[o] + dx;
            sy = s_sy0[o] + dy;
            slot = 2u * dy + dx;
            g = s_gid[o];
            how = s_sw[o] >> 30;  // 1: hitmask, 0: projection's masks, 2: entry_mask
            r = s_rect[o];
            hm = s_hm[o];
        }
        uint32_t mask = entry_mask(valid && how == 2u, g, r, hm, sx * kSuperW, sy * kSuperH, T, sc, lane, s_big[warp]);
        if (valid && how == 1u)
            mask = super_mask_from_hits(hm, r.x & 0xffffu, r.x >> 16, r.y & 0xffffu, r.y >> 16, sx, sy);
        else if (valid && how == 0u)
            mask = smask_slot(s_sm[o], slot);
        const unsigned long long pos = out + k;
        if (valid && pos < (unsigned long long)capacity) {
            const uint32_t key = s_base[o] + sy * s_SX[o] + sx;
            ck[pos] = key;
            sc.vals[0][pos] = (uint32_t)pos;
            gidx[pos] = g;
            gmask[pos] = mask;
            for (int p = 0; p < passes; ++p)
                atomicAdd(&s_hist[p][(key >> (p * kRadixBits)) & (p == passes - 1 ? last_mask : kRadix - 1)], 1u);
        }
    }
    // the sort's digit totals: this CTA's counts added into its partial copy (zeroed before)
    __syncthreads();
    uint32_t* copy = sc.digit_totals + (blockIdx.x % kTotalCopies) * (kMaxPasses * kRadix);
    for (int k = t; k < passes * kRadix; k += kProjBlock) {
        const uint32_t v = (&s_hist[0][0])[k];
        if (v) atomicAdd(&copy[k], v);
    }
}

// ---------------------------------------------------------------------------------------------
// K4: radix sort
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ uint64_t kept_pairs(const Scratch& sc, int64_t capacity) {
    const unsigned long long P = *sc.pair_count;
    return P < (unsigned long long)capacity ? P : (unsigned long long)capacity;
}

// digit totals of every pass (digits from bit first_shift up) in one read of the keys, added into
// the partial copy of the CTA
template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads)
k_digit_totals(int64_t capacity, int first_shift, int passes, uint32_t last_mask, const KeyT* __restrict__ keys,
               Scratch sc) {
    pdl_begin();
    __shared__ uint32_t h[kMaxPasses][kRadix];
    for (int k = threadIdx.x; k < kMaxPasses * kRadix; k += kSortThreads) (&h[0][0])[k] = 0;
    __syncthreads();
    const uint64_t P = kept_pairs(sc, capacity);
    for (uint64_t k = (uint64_t)blockIdx.x * kSortThreads + threadIdx.x; k < P;
         k += (uint64_t)gridDim.x * kSortThreads) {
        const unsigned long long key = keys[k];
        for (int p = 0; p < passes; ++p)
            atomicAdd(&h[p][(key >> (first_shift + p * kRadixBits)) & (p == passes - 1 ? last_mask : kRadix - 1)], 1u);
    }
    __syncthreads();
    uint32_t* copy = sc.digit_totals + (blockIdx.x % kTotalCopies) * (kMaxPasses * kRadix);
    for (int k = threadIdx.x; k < passes * kRadix; k += kSortThreads) {
        const uint32_t v = (&h[0][0])[k];
        if (v) atomicAdd(&copy[k], v);
    }
}

// One pass of the sort in one launch (decoupled look-back): a CTA takes the next tile of
// kSortThreads x kItems keys from a ticket (so every tile before it belongs to a CTA already
// running), counts its keys per digit in shared memory and publishes those counts at once, so the
// tiles after it can add them up before it has finished.  It then ranks its keys by the pass's
// digit (per 32 consecutive keys the lanes of equal digit from one ballot per digit bit, warp
// prefixes per digit) and adds up the counts of the tiles before it by walking back until a tile
// that has published its inclusive prefix.  Each wait on a tile that has not published yet is
// bounded: past kSpinLimit polls (about a second) the CTA records kStatusTimeout, raises the sort's
// abort word, which ends every other wait at once, and leaves its keys unwritten.  The keys are
// then reordered by digit in shared memory and each digit's run written to its global offset
// (digits of smaller value from the pass's totals + the run of the tiles before), so the global
// writes are contiguous runs.
//
// Look-back words: value | flag << 30, flag 1 = the tile's own count, 2 = inclusive prefix of the
// tiles up to it; 0 = not yet published (the region is cleared before every sort).
constexpr uint32_t kLbCount = 1u << 30, kLbPrefix = 2u << 30, kLbValue = (1u << 30) - 1u;
constexpr int kSpinLimit = 1 << 20;  // with the back-off below, about half a second
constexpr int kLbWindow = 8;
constexpr int kDigitWarps = kRadix / 32;  // the warps whose threads own one digit each

// named barrier of the digit warps (the first kRadix threads); barrier 0 is __syncthreads
__device__ __forceinline__ void digit_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kRadix) : "memory"); }

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename KeyT, int kItems, int kThreads = kSortThreads>
constexpr size_t scatter_smem() { return (sizeof(KeyT) + sizeof(uint32_t)) * kThreads * kItems; }

// kThreads = kRadix or a multiple of it: with more threads than digits each warp ranks fewer keys
// and only the first kRadix threads take the per-digit steps (their own named barrier)
template <typename KeyT, int kItems, int kThreads = kSortThreads>
__global__ void __launch_bounds__(kThreads)
k_onesweep(int64_t capacity, int pass, int shift, uint32_t dmask, int sb_max, const KeyT* __restrict__ kin,
           const uint32_t* __restrict__ vin, KeyT* __restrict__ kout, uint32_t* __restrict__ vout, Scratch sc) {
    pdl_begin();
    static_assert(kThreads % kRadix == 0, "whole digit warps");
    constexpr int kWarps = kThreads / 32;
    constexpr int kTile = kThreads * kItems;            // keys per CTA
    constexpr int kWarpItems = kTile / kWarps;          // contiguous keys per warp
    constexpr int kRounds = kWarpItems / 32;            // == kItems
    extern __shared__ __align__(16) unsigned char s_dyn[];
    KeyT* s_keys = reinterpret_cast<KeyT*>(s_dyn);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_dyn + sizeof(KeyT) * kTile);
    __shared__ uint32_t s_wh[kWarps][kRadix];      // per-warp digit counts, then warp prefixes
    __shared__ uint32_t s_gofs[kRadix];            // global offset of this tile's run of digit d
    __shared__ uint32_t s_bstart[kRadix];          // start of digit d inside the CTA's reordering
    __shared__ uint32_t s_part[kDigitWarps];
    __shared__ uint32_t s_hist[kRadix];            // the tile's count of digit d
    __shared__ uint32_t s_tile;
    uint32_t* head = sc.sort_hist;  // [0] abort word, [1 + pass] ticket of the pass, then the look-back
    uint32_t* lb = sc.sort_hist + kLookbackHead + (size_t)pass * kRadix * sb_max;
    const uint32_t nblk = *sc.sort_blocks;
    if (threadIdx.x == 0) s_tile = atomicAdd(&head[1 + pass], 1u);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kWarps * kRadix; k += kThreads) (&s_wh[0][0])[k] = 0;
    if (threadIdx.x < kRadix) s_hist[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= nblk) return;
    const uint64_t P = kept_pairs(sc, capacity);
    const uint64_t cbase = (uint64_t)tile * kTile;
    const uint64_t wbase = cbase + (uint64_t)warp * kWarpItems;
    const unsigned lt = (1u << lane) - 1u;
    KeyT key[kRounds];
    uint32_t val[kRounds];
    uint32_t dr[kRounds];  // digit | warp-local rank << 8
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
        const bool valid = idx < P;
        key[r] = valid ? kin[idx] : (KeyT)0;
        val[r] = valid ? vin[idx] : 0u;
    }
    // the tile's digit counts, published before the ranking
#pragma unroll
    for (int r = 0; r < kRounds; ++r)
        if (wbase + (uint64_t)r * 32 + lane < P) atomicAdd(&s_hist[(uint32_t)(key[r] >> shift) & dmask], 1u);
    __syncthreads();
    uint32_t* const mine = lb + (size_t)tile * kRadix + (threadIdx.x & (kRadix - 1));
    if (threadIdx.x < kRadix) st_relaxed(mine, (tile == 0 ? kLbPrefix : kLbCount) | s_hist[threadIdx.x]);
    const int nbits = __popc(dmask);  // dmask = 2^bits - 1: higher digit bits are zero
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
        const bool valid = idx < P;
        const uint32_t d = valid ? (uint32_t)(key[r] >> shift) & dmask : 0u;
        // lanes holding the same digit: one ballot per digit bit (and one for validity)
        unsigned peers = __ballot_sync(kFull, valid);
        if (!valid) peers = ~peers;
#pragma unroll
        for (int b = 0; b < kRadixBits; ++b) {
            if (b >= nbits) break;  // warp-uniform
            const bool bit = (d >> b) & 1u;
            const unsigned bal = __ballot_sync(kFull, bit);
            peers &= bit ? bal : ~bal;
        }
        uint32_t before = 0;
        if (valid) before = s_wh[warp][d];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) s_wh[warp][d] = before + __popc(peers);
        __syncwarp();
        dr[r] = valid ? (d | ((before + __popc(peers & lt)) << 8)) : 0xffffffffu;
    }
    __syncthreads();
    if (threadIdx.x < kRadix) {  // thread = digit: warp prefixes, the tile's count of the digit, its look-back
        const int d = threadIdx.x;
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t cnt = s_wh[w][d];
            s_wh[w][d] = acc;
            acc += cnt;
        }
        uint32_t before = 0;  // keys of digit d in the tiles before this one
        if (tile != 0) {
            // kLbWindow predecessors per round, loaded together: the walk over tiles that have
            // published only their count costs one memory latency per window, not per tile
            int spins = 0;
            int64_t t = (int64_t)tile - 1;
            while (t >= 0) {
                uint32_t w[kLbWindow];
#pragma unroll
                for (int k = 0; k < kLbWindow; ++k) w[k] = t - k >= 0 ? ld_relaxed(lb + (size_t)(t - k) * kRadix + d) : kLbPrefix;
                int k = 0;
                bool found = false;
#pragma unroll
                for (; k < kLbWindow; ++k) {
                    const uint32_t flag = w[k] & ~kLbValue;
                    if (flag == 0u) break;  // tile t - k has not published yet
                    before += w[k] & kLbValue;
                    if (flag == kLbPrefix) {
                        found = true;
                        break;
                    }
                }
                if (found) break;
                t -= k;
                if (k == kLbWindow) continue;
                // wait (bounded) for tile t, then take the next window from it
                while ((ld_relaxed(lb + (size_t)t * kRadix + d) & ~kLbValue) == 0u) {
                    if (++spins > kSpinLimit) {
                        atomicOr(sc.status, kStatusTimeout);
                        st_relaxed(head, 1u);
                        break;
                    }
                    if ((spins & 63) == 0 && ld_relaxed(head) != 0u) break;  // another wait ran out
                    __nanosleep(64);
                }
                if (ld_relaxed(head) != 0u) break;
            }
            st_relaxed(mine, kLbPrefix | (before + acc));
        }
        // offset of digit d in the pass's output: all keys of smaller digits + the tiles before
        const uint32_t* tot = sc.digit_totals + pass * kRadix;
        uint32_t all = 0;
#pragma unroll
        for (int cpy = 0; cpy < kTotalCopies; ++cpy) all += tot[(size_t)cpy * kMaxPasses * kRadix + d];
        uint32_t incl_all = all, incl = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ta = __shfl_up_sync(kFull, incl_all, o), tb = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) {
                incl_all += ta;
                incl += tb;
            }
        }
        if (lane == 31) s_part[warp] = incl_all;
        digit_sync();
        uint32_t wpre = 0;
#pragma unroll
        for (int w = 0; w < kDigitWarps; ++w) wpre += w < warp ? s_part[w] : 0u;
        s_gofs[d] = wpre + incl_all - all + before;
        digit_sync();
        if (lane == 31) s_part[warp] = incl;  // the tile's own digit counts, for its reordering
        digit_sync();
        wpre = 0;
#pragma unroll
        for (int w = 0; w < kDigitWarps; ++w) wpre += w < warp ? s_part[w] : 0u;
        s_bstart[d] = wpre + incl - acc;
    }
    __syncthreads();
    if (ld_relaxed(head) != 0u) return;  // a wait ran out: the pass is abandoned (status recorded)
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        if (dr[r] != 0xffffffffu) {
            const uint32_t d = dr[r] & 0xffu;
            const uint32_t pos = s_bstart[d] + s_wh[warp][d] + (dr[r] >> 8);
            if (pos < (uint32_t)kTile) {
                s_keys[pos] = key[r];
                s_vals[pos] = val[r];
            } else {
                atomicOr(sc.status, kStatusInternal);
            }
        }
    }
    __syncthreads();
    const uint32_t count = (uint32_t)min((uint64_t)kTile, P - cbase);
    for (uint32_t p = threadIdx.x; p < count; p += kThreads) {
        const KeyT k = s_keys[p];
        const uint32_t d = (uint32_t)(k >> shift) & dmask;
        const uint64_t dst = (uint64_t)s_gofs[d] + (p - s_bstart[d]);
        if (dst < P) {
            kout[dst] = k;
            vout[dst] = s_vals[p];
        } else {
            atomicOr(sc.status, kStatusInternal);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// K5: tile ranges [first, last + 1) from the sorted keys (ranges pre-zeroed)
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_ranges(int64_t capacity, uint32_t tiles, const uint32_t* __restrict__ keys, Scratch sc) {
    pdl_begin();
    const uint64_t P = kept_pairs(sc, capacity);
    // four consecutive keys per thread step (one 16-byte load), with the neighbours either side
    for (uint64_t k0 = ((uint64_t)blockIdx.x * 256 + threadIdx.x) * 4; k0 < P; k0 += (uint64_t)gridDim.x * 1024) {
        uint32_t t[6];
        t[0] = k0 > 0 ? keys[k0 - 1] : 0xffffffffu;
        if (k0 + 4 <= P) {
            const uint4 q = *reinterpret_cast<const uint4*>(keys + k0);
            t[1] = q.x;
            t[2] = q.y;
            t[3] = q.z;
            t[4] = q.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) t[1 + j] = k0 + j < P ? keys[k0 + j] : 0xffffffffu;
        }
        t[5] = k0 + 4 < P ? keys[k0 + 4] : 0xffffffffu;
#pragma unroll
        for (int j = 1; j <= 4; ++j) {
            const uint64_t k = k0 + j - 1;
            if (k >= P) break;
            if (t[j] >= tiles) {
                atomicOr(sc.status, kStatusInternal);
                continue;
            }
            if (t[j - 1] != t[j]) sc.ranges[t[j]].x = (uint32_t)k;
            if (t[j + 1] != t[j]) sc.ranges[t[j]].y = (uint32_t)(k + 1);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// K5: fine stage.  The coarse entries of a super-tile, in depth order, are cut into blocks of
// kFineBlock; a block computes each entry's 32-bit mask of reached tiles of the super-tile and its
// per-tile counts; a scan over each super-tile's blocks and one over the super-tiles give every
// (block, tile) its first pair, and the block writes its pairs: entry e of tile x goes after the
// entries of x in earlier blocks, earlier warps and earlier lanes, i.e. in depth order.
// ---------------------------------------------------------------------------------------------
constexpr int kFineThreads = 256;
constexpr int kFineWarps = kFineThreads / 32;
constexpr int kFineRounds = kFineBlock / kFineThreads;  // entries per thread: warp w takes the
                                                        // block's entries [64 w, 64 w + 64), 32 a round
constexpr int kFineGrid = 152 * 8;  // grid-stride over the blocks

// tile grid of super-tile s: its position and the render it belongs to
struct SuperCell {
    uint32_t sx, sy;
    int TX, TY;
    uint32_t tile_base;
};

__device__ __forceinline__ SuperCell super_cell(uint32_t s, int TX, int TY, const RenderDesc* __restrict__ renders,
                                                int R) {
    SuperCell c;
    uint32_t local = s, SX = (uint32_t)((TX + kSuperW - 1) / kSuperW);
    c.TX = TX;
    c.TY = TY;
    c.tile_base = 0;
    if (renders) {  // the last render whose first super-tile is <= s
        int lo = 0, hi = R - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (renders[mid].super_base <= (int64_t)s) lo = mid;
            else hi = mid - 1;
        }
        local = s - (uint32_t)renders[lo].super_base;
        SX = (uint32_t)renders[lo].SX;
        c.TX = renders[lo].TX;
        c.TY = renders[lo].TY;
        c.tile_base = (uint32_t)renders[lo].tile_base;
    }
    c.sy = local / SX;
    c.sx = local - c.sy * SX;
    return c;
}

// One CTA: blocks per super-tile (ceil(entries / kFineBlock)), their exclusive scan into vbase
// (vbase[S] = all blocks) and each block's record binfo[v] = (super-tile, first entry, end entry,
// block index inside the super-tile).
// crange_from: 0 = crange is already filled (k_ranges over the sorted keys); 1 = the sort was one
// pass of the whole super-tile id (S <= 256): crange is the exclusive scan of its digit totals;
// 2 = one super-tile: crange[0] = all kept entries.
__global__ void __launch_bounds__(kScanThreads)
k_block_prefix(int S, int64_t capacity, Scratch sc, int crange_from) {
    pdl_begin();
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (crange_from == 1) {  // S <= 256 (the parameter is the same for every thread)
        const int s = threadIdx.x;
        uint32_t c = 0;
        if (s < kRadix) {
#pragma unroll
            for (int cpy = 0; cpy < kTotalCopies; ++cpy) c += sc.digit_totals[(size_t)cpy * kMaxPasses * kRadix + s];
        }
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        if (s < S) sc.crange[s] = make_uint2(before + incl - c, before + incl);
        __syncthreads();  // s_warp is reused below; crange is read below
    }
    if (crange_from == 2 && threadIdx.x == 0) {
        const unsigned long long Ce = *sc.coarse_count;
        sc.crange[0] = make_uint2(0u, (uint32_t)(Ce < (unsigned long long)capacity ? Ce : (unsigned long long)capacity));
    }
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < S; base += kScanThreads) {
        const int s = base + threadIdx.x;
        uint32_t nb = 0;
        if (s < S) {
            const uint2 cr = sc.crange[s];
            nb = (cr.y - cr.x + kFineBlock - 1) / kFineBlock;
        }
        uint32_t incl = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = s_warp[lane];
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi += t;
            }
            s_warp[lane] = wi - w;
        }
        __syncthreads();
        const uint32_t carry = s_carry;
        const uint32_t first = carry + s_warp[warp] + incl - nb;
        if (s < S) {
            sc.vbase[s] = first;
            const uint2 cr = sc.crange[s];
            for (uint32_t k = 0; k < nb; ++k)
                if (first + k < (uint64_t)capacity / 32)
                    sc.binfo[first + k] = make_uint4((uint32_t)s, cr.x + k * kFineBlock,
                                                     min(cr.x + (k + 1) * kFineBlock, cr.y), k);
        }
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) s_carry = carry + s_warp[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) sc.vbase[S] = s_carry;
}

// Each block's per-tile counts wc[32 v + x] from its entries' masks.
__global__ void __launch_bounds__(kFineThreads)
k_fine_count(int64_t capacity, const uint32_t* __restrict__ cv, const uint32_t* __restrict__ gmask,
             uint32_t* __restrict__ wc, int S, Scratch sc) {
    pdl_begin();
    __shared__ uint32_t s_cw[kFineWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t VB = sc.vbase[S];
    for (uint32_t v = blockIdx.x; v < VB; v += gridDim.x) {
        if ((uint64_t)v >= (uint64_t)capacity / 32) break;  // no slot for the block (capacity status raised)
        const uint4 bi = sc.binfo[v];  // super-tile, first entry, end entry, block of the super-tile
        uint32_t m[kFineRounds];
#pragma unroll
        for (int r = 0; r < kFineRounds; ++r) {
            const uint64_t e = (uint64_t)bi.y + warp * (32 * kFineRounds) + r * 32 + lane;
            m[r] = e < bi.z ? gmask[cv[e]] : 0u;
        }
        uint32_t cnt = 0;
#pragma unroll
        for (int r = 0; r < kFineRounds; ++r) cnt += __popc(warp_transpose(m[r], lane));
        s_cw[warp][lane] = cnt;
        __syncthreads();
        if (warp == 0) {
            uint32_t sum = 0;
#pragma unroll
            for (int w = 0; w < kFineWarps; ++w) sum += s_cw[w][lane];
            wc[32ull * v + lane] = sum;  // 32 v + 31 < capacity
        }
        __syncthreads();
    }
}

// One CTA per super-tile: exclusive scan of its blocks' per-tile counts (in place), the tiles'
// pair counts stt[32 s + x] and the super-tile's pairs ssum[s].  The last CTA then scans the
// super-tiles' pairs into their first pair sbase[s] and sets the pair count.
__global__ void __launch_bounds__(256)
k_seg_scan(int64_t capacity, uint32_t* __restrict__ wc, Scratch sc) {
    pdl_begin();
    __shared__ uint32_t s_part[8][32];
    const int s = blockIdx.x, x = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t v0 = sc.vbase[s], nb = sc.vbase[s + 1] - v0;
    const uint32_t q = (nb + 7) / 8, r0 = min(nb, w * q), r1 = min(nb, r0 + q);
    uint32_t sum = 0;
    for (uint32_t r = r0; r < r1; ++r) {
        const uint64_t idx = 32ull * (v0 + r) + x;
        if (idx < (uint64_t)capacity) sum += wc[idx];
    }
    s_part[w][x] = sum;
    __syncthreads();
    uint32_t run = 0, total = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t p = s_part[k][x];
        run += k < w ? p : 0u;
        total += p;
    }
    for (uint32_t r = r0; r < r1; ++r) {
        const uint64_t idx = 32ull * (v0 + r) + x;
        if (idx < (uint64_t)capacity) {
            const uint32_t c = wc[idx];
            wc[idx] = run;
            run += c;
        }
    }
    if (w == 0) {
        sc.stt[32 * s + x] = total;
        const uint32_t all = __reduce_add_sync(kFull, total);
        if (x == 0) sc.ssum[s] = all;
    }
    if (!last_cta(&sc.bin_ticket[1])) return;
    const unsigned long long P = cta_scan(
        (int)gridDim.x, [&](int k) { return (unsigned long long)__ldcg(&sc.ssum[k]); },
        [&](int k, unsigned long long v) { sc.sbase[k] = (uint32_t)v; });
    if (threadIdx.x == 0) {
        *sc.pair_count = P;
        if (P > *sc.pair_need) *sc.pair_need = P;
        if (P > (unsigned long long)capacity) atomicOr(sc.status, kStatusCapacity);
    }
}

// The pairs of every block (values = canonical indices into out), and the ranges of a super-tile's
// tiles from its first block.  Per warp and round the 32 masks are transposed, so lane x holds the
// set of lanes reaching tile x: its count is one popcount and an entry's rank among them another.
__global__ void __launch_bounds__(kFineThreads)
k_fine_emit(int64_t capacity, int TX, int TY, const uint32_t* __restrict__ cv, const uint32_t* __restrict__ gidx,
            const uint32_t* __restrict__ gmask, const uint32_t* __restrict__ wc, int S, uint32_t* __restrict__ out,
            Scratch sc, const RenderDesc* __restrict__ renders, int R) {
    pdl_begin();
    __shared__ uint32_t s_cw[kFineWarps][32];
    __shared__ uint32_t s_off[kFineWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t VB = sc.vbase[S];
    for (uint32_t v = blockIdx.x; v < VB; v += gridDim.x) {
        if ((uint64_t)v >= (uint64_t)capacity / 32) break;
        const uint4 bi = sc.binfo[v];
        const uint32_t s = bi.x;
        uint32_t g[kFineRounds], m[kFineRounds], col[kFineRounds];
        uint32_t cnt = 0;
#pragma unroll
        for (int r = 0; r < kFineRounds; ++r) {
            const uint64_t e = (uint64_t)bi.y + warp * (32 * kFineRounds) + r * 32 + lane;
            const bool valid = e < bi.z;
            const uint32_t e0 = valid ? cv[e] : 0u;
            g[r] = valid ? gidx[e0] : 0u;
            m[r] = valid ? gmask[e0] : 0u;
        }
#pragma unroll
        for (int r = 0; r < kFineRounds; ++r) {
            col[r] = warp_transpose(m[r], lane);  // lanes whose entry of round r reaches tile `lane`
            cnt += __popc(col[r]);
        }
        s_cw[warp][lane] = cnt;
        __syncthreads();
        if (warp == 0) {
            const uint32_t tt = sc.stt[32 * s + lane];
            uint32_t incl = tt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t ts = sc.sbase[s] + incl - tt;  // the tile's first pair
            uint32_t base = ts + wc[32ull * v + lane];
#pragma unroll
            for (int w = 0; w < kFineWarps; ++w) {
                s_off[w][lane] = base;
                base += s_cw[w][lane];
            }
            if (bi.w == 0) {
                const SuperCell c = super_cell(s, TX, TY, renders, R);
                const uint32_t tx = c.sx * kSuperW + (lane % kSuperW), ty = c.sy * kSuperH + (lane / kSuperW);
                if ((int)tx < c.TX && (int)ty < c.TY) {
                    const uint32_t cap = capacity < 0xffffffffll ? (uint32_t)capacity : 0xffffffffu;
                    sc.ranges[c.tile_base + ty * (uint32_t)c.TX + tx] = make_uint2(min(ts, cap), min(ts + tt, cap));
                }
            }
        }
        __syncthreads();
        // each lane writes its entries' pairs: tile x after the warp's earlier entries that reach x
#pragma unroll
        for (int r = 0; r < kFineRounds; ++r) {
            uint32_t mm = m[r];
            const int rounds = __reduce_max_sync(kFull, (uint32_t)__popc(mm));
            for (int it = 0; it < rounds; ++it) {  // warp-uniform
                const int x = mm ? __ffs(mm) - 1 : 0;
                uint32_t earlier = 0;
#pragma unroll
                for (int q = 0; q < r; ++q) earlier += __popc(__shfl_sync(kFull, col[q], x));
                const uint32_t cx = __shfl_sync(kFull, col[r], x);
                if (mm) {
                    const uint64_t pos = (uint64_t)s_off[warp][x] + earlier + __popc(cx & lt);
                    if (pos < (uint64_t)capacity) out[pos] = g[r];
                    mm &= mm - 1u;
                }
            }
        }
        __syncthreads();
    }
}

// Counting sort of the tiles into 128 quarter-octave buckets of their list length, heaviest
// bucket first (only the schedule depends on it, never a result; the order inside a bucket is
// arbitrary).  Above kOrderSmall tiles, two launches over CTAs of kOrderThreads x kOrderItems
// tiles: per-CTA bucket counts
// added into the global counts, whose exclusive scan the last CTA writes as the buckets' cursors;
// then each CTA reserves one range per bucket it holds and scatters its tiles into it.
constexpr int kOrderThreads = 256;
constexpr int kOrderItems = 8;
constexpr int kOrderBuckets = 128;

__device__ __forceinline__ int order_slot(const Scratch& sc, int t) {
    const uint2 r = sc.ranges[t];
    const uint32_t len = r.y - r.x;
    // lengths 0..3 are their own buckets; from 4 on, 4 (l - 1) + the two bits after the leading
    // one (l = floor(log2 len)): monotone in the length, at most 123
    int b = (int)len;
    if (len >= 4) {
        const int l = 31 - __clz(len);
        b = 4 * (l - 1) + (int)((len >> (l - 2)) & 3u);
    }
    return kOrderBuckets - 1 - b;
}

// up to kOrderSmall tiles: both steps in one CTA of 1024 threads (one launch); each thread takes
// a run of (at most 16) consecutive tiles, loads their ranges up front and keeps their buckets
// for the scatter.  Runs, not a stride of 1024: the 32 tiles one warp instruction touches are then
// 16 tiles apart instead of neighbours of similar list length, so fewer of its shared-memory
// atomics fall on the same bucket and serialise
constexpr int kOrderSmallThreads = 1024;
constexpr int kOrderSmall = 16384;
constexpr int kOrderSmallItems = kOrderSmall / kOrderSmallThreads;
__global__ void __launch_bounds__(kOrderSmallThreads) k_tile_order_small(int tiles, Scratch sc) {
    pdl_begin();
    __shared__ uint32_t hist[kOrderBuckets], cursor[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) hist[threadIdx.x] = 0;
    int slot[kOrderSmallItems];
#pragma unroll
    for (int k = 0; k < kOrderSmallItems; ++k) {
        const int t = (int)threadIdx.x * kOrderSmallItems + k;
        slot[k] = t < tiles ? order_slot(sc, t) : -1;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOrderSmallItems; ++k)
        if (slot[k] >= 0) atomicAdd(&hist[slot[k]], 1u);
    __syncthreads();
    cta_scan(kOrderBuckets, [&](int k) { return (unsigned long long)hist[k]; },
             [&](int k, unsigned long long v) { cursor[k] = (uint32_t)v; });
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOrderSmallItems; ++k) {
        if (slot[k] < 0) continue;
        const uint32_t pos = atomicAdd(&cursor[slot[k]], 1u);
        if (pos < (uint32_t)tiles) sc.tile_order[pos] = (uint32_t)((int)threadIdx.x * kOrderSmallItems + k);
        else atomicOr(sc.status, kStatusInternal);
    }
}

__global__ void __launch_bounds__(kOrderThreads) k_tile_hist(int tiles, Scratch sc) {
    pdl_begin();
    __shared__ uint32_t hist[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) hist[threadIdx.x] = 0;
    __syncthreads();
    const int t0 = blockIdx.x * kOrderThreads * kOrderItems;
    for (int k = 0; k < kOrderItems; ++k) {
        const int t = t0 + k * kOrderThreads + threadIdx.x;
        if (t < tiles) atomicAdd(&hist[order_slot(sc, t)], 1u);
    }
    __syncthreads();
    uint32_t* counts = sc.tile_buckets;  // [0, 128): counts, [128, 256): cursors
    if (threadIdx.x < kOrderBuckets && hist[threadIdx.x]) atomicAdd(&counts[threadIdx.x], hist[threadIdx.x]);
    if (!last_cta(&sc.bin_ticket[2])) return;
    cta_scan(kOrderBuckets, [&](int k) { return (unsigned long long)__ldcg(&counts[k]); },
             [&](int k, unsigned long long v) { counts[kOrderBuckets + k] = (uint32_t)v; });
    __syncthreads();
    if (threadIdx.x < kOrderBuckets) counts[threadIdx.x] = 0u;  // zero for the next render
}

__global__ void __launch_bounds__(kOrderThreads) k_tile_scatter(int tiles, Scratch sc) {
    pdl_begin();
    __shared__ uint32_t hist[kOrderBuckets], base[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) hist[threadIdx.x] = 0;
    __syncthreads();
    const int t0 = blockIdx.x * kOrderThreads * kOrderItems;
    int slot[kOrderItems];
    uint32_t rank[kOrderItems];
#pragma unroll
    for (int k = 0; k < kOrderItems; ++k) {
        const int t = t0 + k * kOrderThreads + threadIdx.x;
        slot[k] = t < tiles ? order_slot(sc, t) : -1;
        rank[k] = slot[k] >= 0 ? atomicAdd(&hist[slot[k]], 1u) : 0u;
    }
    __syncthreads();
    uint32_t* cursor = sc.tile_buckets + kOrderBuckets;
    if (threadIdx.x < kOrderBuckets && hist[threadIdx.x]) base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], hist[threadIdx.x]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOrderItems; ++k) {
        const int t = t0 + k * kOrderThreads + threadIdx.x;
        if (slot[k] >= 0) {
            const uint32_t pos = base[slot[k]] + rank[k];
            if (pos < (uint32_t)tiles) sc.tile_order[pos] = (uint32_t)t;
            else atomicOr(sc.status, kStatusInternal);
        }
    }
}

}  // namespace

// a pass reorders a whole CTA tile of keys in dynamic shared memory (32 KB with 4096 32-bit keys,
// 48 KB with 4096 64-bit keys)
template <typename KeyT, int kItems, int kThreads = kSortThreads>
void enable_scatter_smem() {
    static bool done = [] {
        cudaFuncSetAttribute(k_onesweep<KeyT, kItems, kThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem<KeyT, kItems, kThreads>());
        return true;
    }();
    (void)done;
}

// LSD passes over bits [first_shift, first_shift + bits) of the keys in keys[0] / keys[1] (viewed
// as KeyT), 8 bits a pass (the last pass takes what is left: bits above the range never take part),
// CTA tiles of kThreads x kItems keys: the digit totals of every pass in one read of the keys,
// then one launch per pass.  Returns the launches and leaves the sorted buffer's index in *out_buf.
// bits of a super-tile id (the coarse sort's key width)
static int super_bits(int64_t supers) {
    int bits = 0;
    while ((1ll << bits) < (long long)supers) ++bits;
    return bits;
}

// cleared: the look-back words (and, unless totals_ready, the digit totals) are already zero.
template <typename KeyT, int kItems, int kThreads = kSortThreads>
int sort_passes(int64_t capacity, int first_shift, int bits, const Scratch& sc, cudaStream_t s, int* out_buf,
                bool totals_ready = false, bool cleared = false) {
    constexpr int kTile = kThreads * kItems;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    const uint32_t last_mask = passes > 0 ? (uint32_t)((1u << (bits - kRadixBits * (passes - 1))) - 1u) : 0u;
    const int sb_max = (int)((capacity + kTile - 1) / kTile);
    // the totals read every key once: one CTA per 1024 keys, at most 8 per SM
    const int64_t want = (capacity + 1023) / 1024;
    const int total_blocks = (int)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
    int buf = 0;
    *out_buf = 0;
    if (sb_max <= 0 || passes <= 0) return 0;
    enable_scatter_smem<KeyT, kItems, kThreads>();
    KeyT* k[2] = {reinterpret_cast<KeyT*>(sc.keys[0]), reinterpret_cast<KeyT*>(sc.keys[1])};
    // abort word, tickets and the look-back words of every pass start cleared
    if (!cleared) cudaMemsetAsync(sc.sort_hist, 0, sizeof(uint32_t) * lookback_words(passes, sb_max), s);
    if (!totals_ready) {  // else the kernel that wrote the keys counted their digits
        if (!cleared) cudaMemsetAsync(sc.digit_totals, 0, sizeof(uint32_t) * kTotalWords, s);
        launch_pdl(k_digit_totals<KeyT>, dim3(total_blocks), dim3(kSortThreads), 0, s, capacity, first_shift, passes,
                   last_mask, (const KeyT*)k[0], sc);
    }
    for (int p = 0; p < passes; ++p) {
        const int shift = first_shift + p * kRadixBits;
        const uint32_t dmask = p == passes - 1 ? last_mask : (uint32_t)(kRadix - 1);
        launch_pdl(k_onesweep<KeyT, kItems, kThreads>, dim3(sb_max), dim3(kThreads), scatter_smem<KeyT, kItems, kThreads>(),
                   s, capacity, p, shift, dmask, sb_max, (const KeyT*)k[buf], (const uint32_t*)sc.vals[buf], k[buf ^ 1],
                   sc.vals[buf ^ 1], sc);
        buf ^= 1;
    }
    *out_buf = buf;
    return (totals_ready ? 0 : 1) + passes;
}

// One radix-sort pass over three tiles of the pair buffers, the first never published: the ticket starts at
// 1, so tile 1 waits on tile 0 until its bound runs out (failure-detection self-test).
__global__ void k_selftest_setup(Scratch sc) {
    *sc.pair_count = 3ull * kSortTile;
    *sc.sort_blocks = 3u;
    sc.sort_hist[1] = 1u;  // the pass's ticket: tile 0 is never taken
}

int launch_timeout_selftest(int64_t capacity, const Scratch& sc, cudaStream_t s) {
    if (capacity < 3 * (int64_t)kSortTile) return 0;
    enable_scatter_smem<uint32_t, kSortItems>();
    const int sb_max = (int)((capacity + kSortTile - 1) / kSortTile);
    cudaMemsetAsync(sc.digit_totals, 0, sizeof(uint32_t) * kTotalWords, s);
    cudaMemsetAsync(sc.sort_hist, 0, sizeof(uint32_t) * lookback_words(1, sb_max), s);
    k_selftest_setup<<<1, 1, 0, s>>>(sc);
    uint32_t* k0 = reinterpret_cast<uint32_t*>(sc.keys[0]);
    uint32_t* k1 = reinterpret_cast<uint32_t*>(sc.keys[1]);
    k_onesweep<uint32_t, kSortItems><<<2, kSortThreads, scatter_smem<uint32_t, kSortItems>(), s>>>(
        capacity, 0, 0, kRadix - 1, sb_max, k0, sc.vals[0], k1, sc.vals[1], sc);
    return 2;
}

int launch_tile_order(int tiles, const Scratch& sc, cudaStream_t s) {
    if (tiles <= 0) return 0;
    if (tiles <= kOrderSmall) {
        launch_pdl(k_tile_order_small, dim3(1), dim3(kOrderSmallThreads), 0, s, tiles, sc);
        return 1;
    }
    const int blocks = (tiles + kOrderThreads * kOrderItems - 1) / (kOrderThreads * kOrderItems);
    launch_pdl(k_tile_hist, dim3(blocks), dim3(kOrderThreads), 0, s, tiles, sc);
    launch_pdl(k_tile_scatter, dim3(blocks), dim3(kOrderThreads), 0, s, tiles, sc);
    return 2;
}

int launch_depth_sort(int64_t n, const Scratch& sc, cudaStream_t s, const uint32_t** perm, bool cleared) {
    Scratch d = sc;
    d.keys[0] = sc.dkeys[0];
    d.keys[1] = sc.dkeys[1];
    d.vals[0] = sc.dvals[0];
    d.vals[1] = sc.dvals[1];
    d.sort_hist = sc.dhist;
    d.digit_totals = sc.dtotals;
    d.pair_count = sc.dcount;
    d.sort_blocks = sc.dblocks;
    int buf = 0;
    const int launched = sort_passes<uint32_t, kDepthItems, kDepthThreads>(n, 0, 32, d, s, &buf, false, cleared);
    *perm = sc.dvals[buf];
    return launched;
}

int launch_bin_count(int64_t n, int64_t supers, int64_t capacity, const uint32_t* perm, const Scratch& sc,
                     cudaStream_t s, bool cleared) {
    const int64_t nbk = (n + kProjBlock - 1) / kProjBlock;
    const int nb = (int)((nbk + kCountItems - 1) / kCountItems);
    if (!cleared) cudaMemsetAsync(sc.pair_count, 0, sizeof(unsigned long long), s);
    launch_pdl(k_coarse_counts, dim3(nb > 0 ? nb : 1), dim3(kProjBlock), 0, s, n, capacity, supers, perm, sc);
    return 1;
}

int launch_bin_lists(int64_t n, int TX, int TY, int T, int64_t tiles, int64_t supers, int64_t capacity,
                     const uint32_t* perm, const Scratch& sc, cudaStream_t s, int* out_buf, const RenderDesc* renders,
                     int R, bool cleared) {
    const int nb = (int)((n + kProjBlock - 1) / kProjBlock);
    int launched = 0;
    *out_buf = 1;
    // canonical index and reach mask of coarse entry e0 in the upper halves of the key buffers (the
    // coarse keys are 32-bit: the sort uses the lower halves)
    uint32_t* gidx = reinterpret_cast<uint32_t*>(sc.keys[0]) + capacity;
    uint32_t* gmask = reinterpret_cast<uint32_t*>(sc.keys[1]) + capacity;
    if (!cleared) cudaMemsetAsync(sc.ranges, 0, sizeof(uint2) * (size_t)tiles, s);
    if (capacity <= 0 || supers <= 0) return 0;
    const int bits = super_bits(supers);
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    const uint32_t last_mask = passes > 0 ? (uint32_t)((1u << (bits - kRadixBits * (passes - 1))) - 1u) : 0u;
    if (!cleared) cudaMemsetAsync(sc.digit_totals, 0, sizeof(uint32_t) * kTotalWords, s);
    if (nb > 0) {
        launch_pdl(k_coarse_emit, dim3(nb), dim3(kProjBlock), 0, s, n, (TX + kSuperW - 1) / kSuperW, T, capacity, perm,
                   sc, gidx, gmask, passes, last_mask, renders, R);
        ++launched;
    }
    // the coarse entries arrive in depth order: a stable sort by super-tile keeps it in each
    // super-tile (its count and CTA count are the coarse stage's, its digit totals the emission's)
    Scratch cs = sc;
    cs.pair_count = sc.coarse_count;
    int cb = 0;
    launched += sort_passes<uint32_t, kCoarseItems, kCoarseThreads>(capacity, 0, bits, cs, s, &cb, true, cleared);
    int crange_from = passes == 0 ? 2 : 1;
    if (passes > 1) {  // the super-tiles' ranges from the sorted keys
        if (!cleared) cudaMemsetAsync(sc.crange, 0, sizeof(uint2) * (size_t)supers, s);
        cs.ranges = sc.crange;
        launch_pdl(k_ranges, dim3(152 * 8), dim3(256), 0, s, capacity, (uint32_t)supers,
                   reinterpret_cast<const uint32_t*>(sc.keys[cb]), cs);
        ++launched;
        crange_from = 0;
    }
    launch_pdl(k_block_prefix, dim3(1), dim3(kScanThreads), 0, s, (int)supers, capacity, sc, crange_from);
    // block counts over the sorted coarse keys (read by k_ranges before)
    uint32_t* wc = reinterpret_cast<uint32_t*>(sc.keys[cb]);
    const uint32_t* cv = sc.vals[cb];
    launch_pdl(k_fine_count, dim3(kFineGrid), dim3(kFineThreads), 0, s, capacity, cv, gmask, wc, (int)supers, sc);
    launch_pdl(k_seg_scan, dim3((unsigned)supers), dim3(256), 0, s, capacity, wc, sc);
    launch_pdl(k_fine_emit, dim3(kFineGrid), dim3(kFineThreads), 0, s, capacity, TX, TY, cv, gidx, gmask, wc, (int)supers,
               sc.vals[cb ^ 1], sc, renders, R);
    *out_buf = cb ^ 1;
    return launched + 4;
}

ZeroPlan render_zero_plan(const Scratch& sc, int64_t n, int64_t tiles, int64_t supers, int64_t capacity) {
    ZeroPlan z{};
    auto add = [&](void* p, size_t words) {
        if (p && words > 0 && z.count < kZeroRegions) {
            z.p[z.count] = static_cast<uint32_t*>(p);
            z.words[z.count] = (uint32_t)words;
            ++z.count;
        }
    };
    // depth sort: 4 passes over ceil(n / kDepthTile) tiles, its digit totals
    add(sc.dhist, lookback_words(32 / kRadixBits, (n + kDepthTile - 1) / kDepthTile));
    add(sc.dtotals, kTotalWords);
    add(sc.pair_count, 2);
    add(sc.ranges, 2 * (size_t)tiles);
    // coarse stage: its digit totals, its sort's look-back words, the super-tiles' ranges
    add(sc.digit_totals, kTotalWords);
    if (capacity > 0 && supers > 0) {
        const int passes = (super_bits(supers) + kRadixBits - 1) / kRadixBits;
        add(sc.sort_hist, lookback_words(passes, (capacity + kSortTile - 1) / kSortTile));
        if (passes > 1) add(sc.crange, 2 * (size_t)supers);
    }
    add(sc.l1_acc, 6);  // the forward's fused L1 sums and ticket
    return z;
}

void clear_zero_plan(const ZeroPlan& z, cudaStream_t s) {
    for (int r = 0; r < z.count; ++r) cudaMemsetAsync(z.p[r], 0, sizeof(uint32_t) * z.words[r], s);
}

int launch_radix_sort_only(int64_t capacity, int key_bits, const Scratch& sc, cudaStream_t s,
                           int* out_buf) {
    return sort_passes<unsigned long long, kSortItems>(capacity, 0, key_bits, sc, s, out_buf);
}

}  // namespace pgs
