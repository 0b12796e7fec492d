// pn_order.cu -- spatial order of the star slots for the packed pair kernel.
//
// The packed pair kernel's work unit is a (target block, source tile) pair.
// When the stars of a block and those of a tile each lie close together in
// space, a unit whose two bounding boxes are far apart can form the pair
// separation from the high single-precision parts of the positions alone
// (k_fused_packed states the criterion and the error bound).  This file puts
// every cluster's star slots in the order of a Hilbert curve, each
// evaluation, from that evaluation's positions:
//
//   key      21-bit Hilbert index of u = d / (|d| + s), quantised to 128 cells
//            per axis (d the hole-relative position from the staged record,
//            s the cluster's mean |d|), so that cells are small near the hole
//            and grow outwards with the falling density; padding slots take
//            the largest key and stay last.  Consecutive cells of a Hilbert
//            curve are neighbours (a Morton curve jumps), which keeps runs of
//            128 sorted stars compact.
//   sort     stable least-significant-digit radix sort, kSortPasses passes of
//            kSortBits bits, within each cluster's slot range: digit counts
//            per 512-slot block, a per-cluster scan of the counts, a stable
//            block scatter.  No atomics decide an order, so the permutation
//            (and every sum taken in it) depends on the positions alone.
//   permute  staged records in sorted order, ssrec[k] = srec[perm[k]], and
//            per tile of kPackTile sorted sources the box of the high parts
//            of d and the largest |d|.
//
// Any permutation gives the same sums up to rounding; the order only decides
// how many units qualify for the cheaper pair body.
#include "pn_device.cuh"

namespace pn {

constexpr int kSortBlock = 512;            // slots per sort block (clusters are padded to kPad)
constexpr int kSortBits = 7;
constexpr int kSortBins = 1 << kSortBits;
constexpr int kSortPasses = 3;             // 21-bit keys
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kScanGroups = 8;             // block groups per digit in k_sort_scan
constexpr unsigned kKeyPad = (1u << (kSortBits * kSortPasses)) - 1u;

static_assert(kPad % kSortBlock == 0, "sort blocks must not straddle clusters");
static_assert(kSortBlock % kGlueThreads == 0, "sort blocks cover whole glue blocks");

constexpr int kCellBits = 7;               // cells per axis: 2^kCellBits
static_assert(3 * kCellBits == kSortBits * kSortPasses, "one key bit per sort bit");

// Spreads the low 7 bits of v to every third bit (bit i -> bit 3 i).
__device__ __forceinline__ unsigned spread3(unsigned v)
{
    v &= 0x7fu;
    v = (v | (v << 8)) & 0x0000f00fu;
    v = (v | (v << 4)) & 0x000c30c3u;
    v = (v | (v << 2)) & 0x00249249u;
    return v;
}

__device__ __forceinline__ unsigned quantise(float d, float inv_len)
{
    // u in (-1, 1) -> cell 0..127
    const float u = d * inv_len;
    const int q = (int)floorf((u + 1.0f) * 64.0f);
    return (unsigned)(q < 0 ? 0 : (q > 127 ? 127 : q));
}

// Hilbert index of the cell (X[0], X[1], X[2]), each in [0, 2^kCellBits):
// Skilling's transform of the axes into the "transposed" index (J. Skilling,
// Programming the Hilbert curve, AIP Conf. Proc. 707, 381 (2004)) -- undo
// the excess work level by level, then Gray-code -- whose bits, interleaved
// from the top level down with X[0] first, are the index.
__device__ __forceinline__ unsigned hilbert3(unsigned X0, unsigned X1, unsigned X2)
{
    unsigned X[3] = {X0, X1, X2};
    constexpr unsigned M = 1u << (kCellBits - 1);
#pragma unroll
    for (unsigned Q = M; Q > 1; Q >>= 1) {
        const unsigned P = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;                              // invert the low bits
            } else {
                const unsigned t = (X[0] ^ X[i]) & P;   // exchange them
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    unsigned t = 0;
#pragma unroll
    for (unsigned Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q)
            t ^= Q - 1;
    return (spread3(X[0] ^ t) << 2) | (spread3(X[1] ^ t) << 1) | spread3(X[2] ^ t);
}

// Hilbert key of slot t from its staged record (F0 = (-hx, -hx, -hy, -hy),
// F1 = (-hz, -hz, m, m)); padding slots (past the cluster's stars) get kKeyPad.
__device__ __forceinline__ unsigned slot_key(const Clu &C, int64_t t, const float4 *__restrict__ srec,
                                             float s)
{
    if (t - C.slot0 >= C.ns)
        return kKeyPad;
    const float4 F0 = srec[t * kFwdVals], F1 = srec[t * kFwdVals + 1];
    const float dx = -F0.x, dy = -F0.z, dz = -F1.x;
    const float inv = 1.0f / (sqrtf(dx * dx + dy * dy + dz * dz) + s);
    return hilbert3(quantise(dx, inv), quantise(dy, inv), quantise(dz, inv));
}

__device__ __forceinline__ const Clu &block_cluster(const Clu *__restrict__ clu,
                                                    const int *__restrict__ blk_clu, int64_t b)
{
    return clu[cluster_of_block(blk_clu, b * (kSortBlock / kGlueThreads))];
}

// Digit counts of sort block b for pass PASS: hist[b][digit].  Pass 0 also
// computes the keys (slot order) into keys[].
template <int PASS>
__global__ void __launch_bounds__(kSortBlock)
k_sort_hist(const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
            const float4 *__restrict__ srec, const double *__restrict__ glob,
            unsigned *__restrict__ keys, int *__restrict__ hist)
{
    __shared__ int h[kSortBins];
    const int64_t b = blockIdx.x;
    const int64_t t = b * kSortBlock + threadIdx.x;
    if (threadIdx.x < kSortBins)
        h[threadIdx.x] = 0;
    __syncthreads();
    unsigned key;
    if (PASS == 0) {
        const Clu &C = block_cluster(clu, blk_clu, b);
        const int k = cluster_of_block(blk_clu, b * (kSortBlock / kGlueThreads));
        const double mean_r = glob[(int64_t)k * kGlobVals + kGlobMeanR] / (double)(C.ns > 0 ? C.ns : 1);
        const float s = mean_r > 1e-30 ? (float)mean_r : 1e-30f;
        key = slot_key(C, t, srec, s);
        keys[t] = key;
    } else {
        key = keys[t];
    }
    atomicAdd(&h[(key >> (kSortBits * PASS)) & (kSortBins - 1)], 1);
    __syncthreads();
    if (threadIdx.x < kSortBins)
        hist[b * kSortBins + threadIdx.x] = h[threadIdx.x];
}

// One block per cluster: turns the digit counts of the cluster's sort blocks
// into scatter offsets, hist[b][d] = slot0 + (keys of the cluster with a
// smaller digit) + (keys with digit d in the cluster's earlier blocks).
__global__ void __launch_bounds__(kSortBins * kScanGroups)
k_sort_scan(const Clu *__restrict__ clu, int *__restrict__ hist)
{
    __shared__ int part[kScanGroups][kSortBins];
    __shared__ int dbase[kSortBins];
    const Clu C = clu[blockIdx.x];
    const int d = threadIdx.x % kSortBins, g = threadIdx.x / kSortBins;
    const int64_t b0 = C.slot0 / kSortBlock, nb = C.ns_pad / kSortBlock;
    const int64_t ch = (nb + kScanGroups - 1) / kScanGroups;
    const int64_t g0 = b0 + g * ch, g1 = (g0 + ch < b0 + nb) ? g0 + ch : b0 + nb;
    int s = 0;
    for (int64_t b = g0; b < g1; ++b)
        s += hist[b * kSortBins + d];
    part[g][d] = s;
    __syncthreads();
    if (g == 0) {
        int run = 0;
        for (int q = 0; q < kScanGroups; ++q) {
            const int c = part[q][d];
            part[q][d] = run;
            run += c;
        }
        dbase[d] = run;               // total of digit d, scanned below
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int q = 0; q < kSortBins; ++q) {
            const int c = dbase[q];
            dbase[q] = run;
            run += c;
        }
    }
    __syncthreads();
    int run = (int)C.slot0 + dbase[d] + part[g][d];
    for (int64_t b = g0; b < g1; ++b) {
        const int c = hist[b * kSortBins + d];
        hist[b * kSortBins + d] = run;
        run += c;
    }
}

// Stable scatter of sort block b for pass PASS: an item's destination is its
// digit's offset plus the number of items of the block before it with the
// same digit (warp ranks by __match_any_sync, then earlier warps' counts).
// Pass 0 reads the slot index itself as the value.
template <int PASS>
__global__ void __launch_bounds__(kSortBlock)
k_sort_scatter(const unsigned *__restrict__ kin, const int *__restrict__ vin,
               const int *__restrict__ hist, unsigned *__restrict__ kout,
               int *__restrict__ vout)
{
    __shared__ int cnt[kSortWarps][kSortBins];
    const int64_t b = blockIdx.x;
    const int64_t t = b * kSortBlock + threadIdx.x;
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int q = threadIdx.x; q < kSortWarps * kSortBins; q += kSortBlock)
        (&cnt[0][0])[q] = 0;
    const unsigned key = kin[t];
    const int val = PASS == 0 ? (int)t : vin[t];
    const unsigned d = (key >> (kSortBits * PASS)) & (kSortBins - 1);
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == __ffs(peers) - 1)
        cnt[w][d] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < kSortBins) {
        int run = 0;
        for (int q = 0; q < kSortWarps; ++q) {
            const int c = cnt[q][threadIdx.x];
            cnt[q][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    const int dest = hist[b * kSortBins + d] + cnt[w][d] + rank;
    kout[dest] = key;
    vout[dest] = val;
}

// Sorted staged records and tile boxes: one block of kPackTile threads per
// tile of sorted sources.  box[2 T] = (min of the high parts of d, 0),
// box[2 T + 1] = (max of the high parts of d, largest |d|).
__global__ void __launch_bounds__(kPackTile)
k_sort_permute(const float4 *__restrict__ srec, const int *__restrict__ perm,
               float4 *__restrict__ ssrec, float4 *__restrict__ box)
{
    static_assert(kPackTile == 64, "two warps per tile");
    __shared__ float red[2][7];
    const int64_t k = (int64_t)blockIdx.x * kPackTile + threadIdx.x;
    const int64_t slot = perm[k];
    const float4 *src = srec + slot * kFwdVals;
    float4 *dst = ssrec + k * kFwdVals;
    float4 r[kFwdVals];
#pragma unroll
    for (int q = 0; q < kFwdVals; ++q)
        r[q] = src[q];
#pragma unroll
    for (int q = 0; q < kFwdVals; ++q)
        dst[q] = r[q];
    float v[7] = {-r[0].x, -r[0].z, -r[1].x, -r[0].x, -r[0].z, -r[1].x, r[7].z};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < 3; ++q)
            v[q] = fminf(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
#pragma unroll
        for (int q = 3; q < 7; ++q)
            v[q] = fmaxf(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
    }
    if (threadIdx.x % 32 == 0)
#pragma unroll
        for (int q = 0; q < 7; ++q)
            red[threadIdx.x / 32][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        box[2 * blockIdx.x] = make_float4(fminf(red[0][0], red[1][0]), fminf(red[0][1], red[1][1]),
                                          fminf(red[0][2], red[1][2]), 0.0f);
        box[2 * blockIdx.x + 1] =
            make_float4(fmaxf(red[0][3], red[1][3]), fmaxf(red[0][4], red[1][4]),
                        fmaxf(red[0][5], red[1][5]), sqrtf(fmaxf(red[0][6], red[1][6])));
    }
}

size_t order_buffer_bytes(int64_t S)
{
    return sizeof(float4) * (size_t)(kFwdVals * S + 2 * (S / kPackTile)) +
           sizeof(unsigned) * 2 * (size_t)S + sizeof(int) * 2 * (size_t)S +
           sizeof(int) * (size_t)(S / kSortBlock) * kSortBins;
}

Order order_of(pn_ctx *c)
{
    Order o;
    char *p = reinterpret_cast<char *>(c->sord);
    const int64_t S = c->S;
    o.ssrec = reinterpret_cast<float4 *>(p);
    p += sizeof(float4) * kFwdVals * S;
    o.box = reinterpret_cast<float4 *>(p);
    p += sizeof(float4) * 2 * (S / kPackTile);
    o.keys = reinterpret_cast<unsigned *>(p);
    p += sizeof(unsigned) * 2 * S;
    o.vals = reinterpret_cast<int *>(p);
    p += sizeof(int) * 2 * S;
    o.hist = reinterpret_cast<int *>(p);
    o.perm = o.vals + S;          // the last pass (2) writes the second half
    return o;
}

// Hilbert order of the current staged records (c->mrec + 5 S, written by the
// prologue in the law-of-cosines layout) and the sorted records and boxes.
cudaError_t launch_spatial_order(pn_ctx *c)
{
    static_assert(kSortPasses == 3, "the pass sequence below ends in the second buffers");
    const Order o = order_of(c);
    const int64_t S = c->S, nb = S / kSortBlock;
    const float4 *srec = c->mrec + 5 * S;
    const int *bc = c->nclu > 1 ? c->blk_clu : nullptr;
    unsigned *ka = o.keys, *kb = o.keys + S;
    int *va = o.vals, *vb = o.vals + S;
    k_sort_hist<0><<<(unsigned)nb, kSortBlock, 0, c->stream>>>(c->d_clu, bc, srec, c->glob, ka, o.hist);
    k_sort_scan<<<c->nclu, kSortBins * kScanGroups, 0, c->stream>>>(c->d_clu, o.hist);
    k_sort_scatter<0><<<(unsigned)nb, kSortBlock, 0, c->stream>>>(ka, nullptr, o.hist, kb, vb);
    k_sort_hist<1><<<(unsigned)nb, kSortBlock, 0, c->stream>>>(c->d_clu, bc, srec, c->glob, kb, o.hist);
    k_sort_scan<<<c->nclu, kSortBins * kScanGroups, 0, c->stream>>>(c->d_clu, o.hist);
    k_sort_scatter<1><<<(unsigned)nb, kSortBlock, 0, c->stream>>>(kb, vb, o.hist, ka, va);
    k_sort_hist<2><<<(unsigned)nb, kSortBlock, 0, c->stream>>>(c->d_clu, bc, srec, c->glob, ka, o.hist);
    k_sort_scan<<<c->nclu, kSortBins * kScanGroups, 0, c->stream>>>(c->d_clu, o.hist);
    k_sort_scatter<2><<<(unsigned)nb, kSortBlock, 0, c->stream>>>(ka, va, o.hist, kb, vb);
    k_sort_permute<<<(unsigned)(S / kPackTile), kPackTile, 0, c->stream>>>(srec, o.perm, o.ssrec, o.box);
    c->launches += 10;
    return cudaGetLastError();
}

}  // namespace pn
