// K2 scan, K3 key emission, K4 radix sort, K5 tile ranges.
//
// The sorted (tile | depth) keys carry the canonical index as their value: this is the
// permutation pi of Eq. 10 ("a GPU sort yields a permutation mapping sorted index i to canonical
// index pi(i)").  Parameters are never reordered; the compositing kernels gather by pi and the
// backward scatters gradients to pi (index-mapped gradient scattering).
//
// key = (tile << 32) | float bits of the camera depth (depth > near > 0, so the bits order like
// the depths); equal keys keep emission order (canonical order), so the sort is the stable sort
// of the pairs.  The Gaussians are first sorted by depth (32-bit depth keys) and the pairs are
// emitted in that order, so the pair sort only has to order the 32-bit tile part stably: the
// pair buffers hold tile ids (uint32), and the full 64-bit key of a sorted pair is
// (tile << 32) | depth bits of its Gaussian.  The number of pairs is known only on the device: every kernel reads it from the
// context's pair counter, and pairs beyond the capacity are not written (the status word records
// the overflow), so no host synchronisation sits between projection and compositing.
//
// The radix sort is least-significant-digit first, 8-bit digits, over the bits that can be
// non-zero (32 depth bits for the Gaussians, ceil(log2 tiles) tile bits for the pairs; the
// caller's low key bits of the 64-bit keys of the allocation-free entry point); the last digit is
// masked to what is left of the bit range.  The digit totals of every pass come from one up-front
// histogram; each pass is then one launch that ranks a tile's keys with warp ballots and finds the
// tile's place by decoupled look-back over the tiles before it (bounded waits, see k_onesweep).
#include "pgs_internal.cuh"

namespace pgs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
static_assert(kSortThreads == kRadix, "one thread per digit in the sort kernels");

// ---------------------------------------------------------------------------------------------
// K2: exclusive scan of the per-CTA tile counts -> pair offsets, total pair count, capacity check
// ---------------------------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads)
k_scan_blocks(int nb, int64_t capacity, Scratch sc) {
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += kScanThreads) {
        const int idx = base + threadIdx.x;
        unsigned long long v = idx < nb ? sc.block_sums[idx] : 0ull;
        unsigned long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_warp[lane];
            unsigned long long wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long t = __shfl_up_sync(kFull, wi, o);
                if (lane >= o) wi += t;
            }
            s_warp[lane] = wi - w;  // exclusive prefix of warp totals
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        if (idx < nb) sc.block_offsets[idx] = carry + s_warp[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) s_carry = carry + s_warp[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long P = s_carry;
        *sc.pair_count = P;
        const unsigned long long kept = P < (unsigned long long)capacity ? P : (unsigned long long)capacity;
        *sc.sort_blocks = (uint32_t)((kept + kSortTile - 1) / kSortTile);
        if (P > (unsigned long long)capacity) atomicOr(sc.status, kStatusCapacity);
    }
}

// per-CTA sums of tiles touched, Gaussians taken in depth order
__global__ void __launch_bounds__(kProjBlock)
k_perm_counts(int64_t n, const uint32_t* __restrict__ perm, Scratch sc) {
    const int64_t i = (int64_t)blockIdx.x * kProjBlock + threadIdx.x;
    const uint32_t count = i < n ? sc.touched[perm[i]] : 0u;
    const uint32_t warp_sum = __reduce_add_sync(kFull, count);
    __shared__ uint32_t s_part[kProjBlock / 32];
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = warp_sum;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < kProjBlock / 32 ? s_part[threadIdx.x] : 0u;
        v = __reduce_add_sync(kFull, v);
        if (threadIdx.x == 0) sc.block_sums[blockIdx.x] = v;
    }
}

// ---------------------------------------------------------------------------------------------
// K3: emit the pairs of one CTA's Gaussians in depth order (ties: canonical order), tiles
// row-major inside each rectangle.  Each warp walks the candidate tiles of its own 32 Gaussians,
// 32 per round (candidate k by lane k mod 32; its Gaussian found by a shuffle binary search over
// the lanes' inclusive rectangle areas), and compacts the reached ones in order with one ballot.
// A warp's output starts after the pairs of the warps before it, known from the Gaussians'
// reached-tile counts, so warps never wait for one another inside the walk.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kProjBlock)
k_emit(int64_t n, int TX, int T, int64_t capacity, const uint32_t* __restrict__ perm, Scratch sc,
       const RenderDesc* __restrict__ renders, int R) {
    __shared__ uint32_t s_x0[kProjBlock], s_y0[kProjBlock], s_w[kProjBlock];
    __shared__ uint32_t s_tx[kProjBlock], s_tbase[kProjBlock];
    __shared__ float s_u[kProjBlock], s_v[kProjBlock], s_ca[kProjBlock], s_cb[kProjBlock], s_cc[kProjBlock];
    __shared__ float s_sx[kProjBlock], s_sy[kProjBlock];
    __shared__ uint32_t s_mask[kProjBlock];
    __shared__ uint32_t s_warp[kProjBlock / 32];
    __shared__ uint32_t s_gid[kProjBlock];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t i = (int64_t)blockIdx.x * kProjBlock + t;
    uint32_t cnt = 0, reached = 0;  // rectangle area, reached tiles
    if (i < n) {
        const uint32_t g = perm[i];
        s_gid[t] = g;
        reached = sc.touched[g];
        if (reached) {
            const uint2 r = sc.rect[g];
            s_x0[t] = r.x & 0xffffu;
            s_y0[t] = r.x >> 16;
            s_w[t] = (r.y & 0xffffu) - (r.x & 0xffffu);
            cnt = s_w[t] * ((r.y >> 16) - (r.x >> 16));
            const float4 p = sc.xyo[g], q = sc.conic[g];
            s_u[t] = p.x;
            s_v[t] = p.y;
            s_ca[t] = q.x;
            s_cb[t] = q.y;
            s_cc[t] = q.z;
            s_sx[t] = __fdiv_rn(q.y, q.x);
            s_sy[t] = __fdiv_rn(q.y, q.z);
            s_mask[t] = sc.hitmask[g];
            s_tx[t] = (uint32_t)TX;
            s_tbase[t] = 0;
            if (renders) {  // batch: item g belongs to the last render whose first item is <= g
                int lo = 0, hi = R - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (renders[mid].item_base <= (int64_t)g) lo = mid;
                    else hi = mid - 1;
                }
                s_tx[t] = (uint32_t)renders[lo].TX;
                s_tbase[t] = (uint32_t)renders[lo].tile_base;
            }
        }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t first = incl - cnt;  // this lane's first candidate in the warp's walk
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t wpairs = __reduce_add_sync(kFull, reached);
    if (lane == 0) s_warp[warp] = wpairs;
    __syncthreads();  // also publishes the lanes' records in shared memory
    uint32_t before = 0;
#pragma unroll
    for (int w = 0; w < kProjBlock / 32; ++w) before += w < warp ? s_warp[w] : 0u;
    const unsigned long long out = sc.block_offsets[blockIdx.x] + before;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t written = 0;
    for (uint32_t b = 0; b < total; b += 32) {  // warp-uniform
        const uint32_t k = b + (uint32_t)lane;
        int lo = 0, hi = 31;  // owner of candidate k: the first lane whose inclusive area exceeds k
#pragma unroll
        for (int step = 0; step < 5; ++step) {
            const int mid = (lo + hi) >> 1;
            const uint32_t im = __shfl_sync(kFull, incl, mid);
            if (lo < hi) {
                if (im > k) hi = mid;
                else lo = mid + 1;
            }
        }
        const uint32_t ofirst = __shfl_sync(kFull, first, lo), oarea = __shfl_sync(kFull, cnt, lo);
        bool hit = false;
        uint32_t tile = 0, gid = 0;
        if (k < total) {  // then the owner's rectangle is not empty
            const int o = warp * 32 + lo;
            const uint32_t local = k - ofirst;
            const uint32_t w = s_w[o];
            const uint32_t dy = local / w, dx = local - dy * w;
            const uint32_t tx = s_x0[o] + dx, ty = s_y0[o] + dy;
            hit = oarea <= 32u ? ((s_mask[o] >> local) & 1u) != 0u
                               : tile_hit(s_u[o], s_v[o], s_ca[o], s_cb[o], s_cc[o], s_sx[o], s_sy[o], (int)tx,
                                          (int)ty, T);
            tile = s_tbase[o] + ty * s_tx[o] + tx;
            gid = s_gid[o];
        }
        const unsigned bal = __ballot_sync(kFull, hit);
        if (hit) {
            const unsigned long long pos = out + written + __popc(bal & lt);
            if (pos < (unsigned long long)capacity) {
                reinterpret_cast<uint32_t*>(sc.keys[0])[pos] = tile;
                sc.vals[0][pos] = gid;
            }
        }
        written += __popc(bal);
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
constexpr int kSortWarps = kSortThreads / 32;

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename KeyT, int kItems>
constexpr size_t scatter_smem() { return (sizeof(KeyT) + sizeof(uint32_t)) * kSortThreads * kItems; }

template <typename KeyT, int kItems>
__global__ void __launch_bounds__(kSortThreads)
k_onesweep(int64_t capacity, int pass, int shift, uint32_t dmask, int sb_max, const KeyT* __restrict__ kin,
           const uint32_t* __restrict__ vin, KeyT* __restrict__ kout, uint32_t* __restrict__ vout, Scratch sc) {
    constexpr int kTile = kSortThreads * kItems;        // keys per CTA
    constexpr int kWarpItems = kTile / kSortWarps;      // contiguous keys per warp
    constexpr int kRounds = kWarpItems / 32;            // == kItems
    extern __shared__ __align__(16) unsigned char s_dyn[];
    KeyT* s_keys = reinterpret_cast<KeyT*>(s_dyn);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_dyn + sizeof(KeyT) * kTile);
    __shared__ uint32_t s_wh[kSortWarps][kRadix];  // per-warp digit counts, then warp prefixes
    __shared__ uint32_t s_gofs[kRadix];            // global offset of this tile's run of digit d
    __shared__ uint32_t s_bstart[kRadix];          // start of digit d inside the CTA's reordering
    __shared__ uint32_t s_part[kSortWarps];
    __shared__ uint32_t s_hist[kRadix];            // the tile's count of digit d
    __shared__ uint32_t s_tile;
    uint32_t* head = sc.sort_hist;  // [0] abort word, [1 + pass] ticket of the pass, then the look-back
    uint32_t* lb = sc.sort_hist + kLookbackHead + (size_t)pass * kRadix * sb_max;
    const uint32_t nblk = *sc.sort_blocks;
    if (threadIdx.x == 0) s_tile = atomicAdd(&head[1 + pass], 1u);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kSortWarps * kRadix; k += kSortThreads) (&s_wh[0][0])[k] = 0;
    s_hist[threadIdx.x] = 0;
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
    uint32_t* const mine = lb + (size_t)tile * kRadix + threadIdx.x;
    st_relaxed(mine, (tile == 0 ? kLbPrefix : kLbCount) | s_hist[threadIdx.x]);
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
    {   // thread = digit: warp prefixes, the tile's count of the digit, its look-back
        const int d = threadIdx.x;
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
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
        __syncthreads();
        uint32_t wpre = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) wpre += w < warp ? s_part[w] : 0u;
        s_gofs[d] = wpre + incl_all - all + before;
        __syncthreads();
        if (lane == 31) s_part[warp] = incl;  // the tile's own digit counts, for its reordering
        __syncthreads();
        wpre = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) wpre += w < warp ? s_part[w] : 0u;
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
    for (uint32_t p = threadIdx.x; p < count; p += kSortThreads) {
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

// the full keys of the sorted pairs, (tile << 32) | depth bits of the pair's Gaussian
__global__ void __launch_bounds__(256)
k_join_keys(int64_t capacity, const uint32_t* __restrict__ tiles, const uint32_t* __restrict__ vals,
            unsigned long long* __restrict__ out, Scratch sc) {
    const uint64_t P = kept_pairs(sc, capacity);
    for (uint64_t k = (uint64_t)blockIdx.x * 256 + threadIdx.x; k < P; k += (uint64_t)gridDim.x * 256)
        out[k] = ((unsigned long long)tiles[k] << 32) | sc.depth_bits[vals[k]];
}

// One CTA: counting sort of the tiles into 128 quarter-octave buckets of their list length,
// heaviest bucket first.  Only the schedule depends on it, never a result.
constexpr int kOrderThreads = 1024;
constexpr int kOrderBuckets = 128;

__global__ void __launch_bounds__(kOrderThreads) k_tile_order(int tiles, Scratch sc) {
    __shared__ uint32_t hist[kOrderBuckets], cursor[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) hist[threadIdx.x] = 0;
    __syncthreads();
    auto slot_of = [&](int t) {
        const uint2 r = sc.ranges[t];
        const uint32_t len = r.y - r.x;
        // lengths 0..3 are their own buckets; from 4 on, 4 (l - 1) + the two bits after the
        // leading one (l = floor(log2 len)): monotone in the length, at most 123
        int b = (int)len;
        if (len >= 4) {
            const int l = 31 - __clz(len);
            b = 4 * (l - 1) + (int)((len >> (l - 2)) & 3u);
        }
        return kOrderBuckets - 1 - b;
    };
    for (int t = threadIdx.x; t < tiles; t += kOrderThreads) atomicAdd(&hist[slot_of(t)], 1u);
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan, 4 buckets per lane
        const int lane = threadIdx.x;
        uint32_t h[4], s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            h[k] = hist[4 * lane + k];
            s += h[k];
        }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        uint32_t run = incl - s;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            cursor[4 * lane + k] = run;
            run += h[k];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += kOrderThreads)
        sc.tile_order[atomicAdd(&cursor[slot_of(t)], 1u)] = (uint32_t)t;
}

}  // namespace

// a pass reorders a whole CTA tile of keys in dynamic shared memory (32 KB with 4096 32-bit keys,
// 48 KB with 4096 64-bit keys)
template <typename KeyT, int kItems>
void enable_scatter_smem() {
    static bool done = [] {
        cudaFuncSetAttribute(k_onesweep<KeyT, kItems>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem<KeyT, kItems>());
        return true;
    }();
    (void)done;
}

// LSD passes over bits [first_shift, first_shift + bits) of the keys in keys[0] / keys[1] (viewed
// as KeyT), 8 bits a pass (the last pass takes what is left: bits above the range never take part),
// CTA tiles of kSortThreads x kItems keys: the digit totals of every pass in one read of the keys,
// then one launch per pass.  Returns the launches and leaves the sorted buffer's index in *out_buf.
template <typename KeyT, int kItems>
int sort_passes(int64_t capacity, int first_shift, int bits, const Scratch& sc, cudaStream_t s, int* out_buf) {
    constexpr int kTile = kSortThreads * kItems;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    const uint32_t last_mask = passes > 0 ? (uint32_t)((1u << (bits - kRadixBits * (passes - 1))) - 1u) : 0u;
    const int sb_max = (int)((capacity + kTile - 1) / kTile);
    // the totals read every key once: one CTA per 1024 keys, at most 8 per SM
    const int64_t want = (capacity + 1023) / 1024;
    const int total_blocks = (int)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
    int buf = 0;
    *out_buf = 0;
    if (sb_max <= 0 || passes <= 0) return 0;
    enable_scatter_smem<KeyT, kItems>();
    KeyT* k[2] = {reinterpret_cast<KeyT*>(sc.keys[0]), reinterpret_cast<KeyT*>(sc.keys[1])};
    cudaMemsetAsync(sc.digit_totals, 0, sizeof(uint32_t) * kTotalWords, s);
    // abort word, tickets and the look-back words of every pass start cleared
    cudaMemsetAsync(sc.sort_hist, 0, sizeof(uint32_t) * (kLookbackHead + (size_t)passes * kRadix * sb_max), s);
    k_digit_totals<KeyT><<<total_blocks, kSortThreads, 0, s>>>(capacity, first_shift, passes, last_mask, k[0], sc);
    for (int p = 0; p < passes; ++p) {
        const int shift = first_shift + p * kRadixBits;
        const uint32_t dmask = p == passes - 1 ? last_mask : (uint32_t)(kRadix - 1);
        k_onesweep<KeyT, kItems><<<sb_max, kSortThreads, scatter_smem<KeyT, kItems>(), s>>>(
            capacity, p, shift, dmask, sb_max, k[buf], sc.vals[buf], k[buf ^ 1], sc.vals[buf ^ 1], sc);
        buf ^= 1;
    }
    *out_buf = buf;
    return 1 + passes;
}

// One pass of the pair sort over three tiles whose first is never published: the ticket starts at
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
    k_tile_order<<<1, kOrderThreads, 0, s>>>(tiles, sc);
    return 1;
}

int launch_depth_sort(int64_t n, const Scratch& sc, cudaStream_t s, const uint32_t** perm) {
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
    const int launched = sort_passes<uint32_t, kDepthItems>(n, 0, 32, d, s, &buf);
    *perm = sc.dvals[buf];
    return launched;
}

int launch_scan_emit(int64_t n, int TX, int T, int64_t capacity, const uint32_t* perm, const Scratch& sc,
                     cudaStream_t s, const RenderDesc* renders, int R) {
    const int nb = (int)((n + kProjBlock - 1) / kProjBlock);
    if (nb > 0) k_perm_counts<<<nb, kProjBlock, 0, s>>>(n, perm, sc);
    k_scan_blocks<<<1, kScanThreads, 0, s>>>(nb, capacity, sc);
    if (nb == 0) return 1;
    k_emit<<<nb, kProjBlock, 0, s>>>(n, TX, T, capacity, perm, sc, renders, R);
    return 3;
}

int launch_sort_ranges(int64_t capacity, int tiles, const Scratch& sc, cudaStream_t s, int* out_buf) {
    int tile_bits = 0;
    while ((1ll << tile_bits) < (long long)tiles) ++tile_bits;
    // the pairs arrive in depth order: a stable sort of their 32-bit tile keys completes it
    int buf = 0;
    int launched = sort_passes<uint32_t, kSortItems>(capacity, 0, tile_bits, sc, s, &buf);
    cudaMemsetAsync(sc.ranges, 0, sizeof(uint2) * (size_t)tiles, s);
    if (capacity > 0) {
        k_ranges<<<152 * 8, 256, 0, s>>>(capacity, (uint32_t)tiles, reinterpret_cast<const uint32_t*>(sc.keys[buf]), sc);
        ++launched;
    }
    *out_buf = buf;
    return launched;
}

int launch_join_keys(int64_t capacity, int buf, const Scratch& sc, cudaStream_t s) {
    if (capacity <= 0) return 0;
    k_join_keys<<<152 * 8, 256, 0, s>>>(capacity, reinterpret_cast<const uint32_t*>(sc.keys[buf]),
                                         sc.vals[buf], sc.keys[buf ^ 1], sc);
    return 1;
}

int launch_radix_sort_only(int64_t capacity, int key_bits, const Scratch& sc, cudaStream_t s,
                           int* out_buf) {
    return sort_passes<unsigned long long, kSortItems>(capacity, 0, key_bits, sc, s, out_buf);
}

}  // namespace pgs
