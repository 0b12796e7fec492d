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
//
// Cost-balanced stream-K workers.  On the spatial order a unit costs more
// when it is near (the full separation) than when it is far, and the near
// units gather in the dense core, so workers of equal unit counts differ in
// cost and the last ones to finish leave the GPU partly idle.  After the
// permutation, every unit gets the FP32-pipe operations per pair of the body
// its block will run (kOpsNear when any warp of the target block is near or
// the unit holds self pairs -- the block's warps meet at every tile -- else
// kOpsFar), and the worker boundaries are cut at equal shares of the total:
//   k_unit_cost      one block per target-block row: costs, in-row prefix,
//                    row total;
//   k_row_scan       prefix over the rows;
//   k_worker_bounds  worker w starts at the first unit whose prefix reaches
//                    w total / G (binary search).
// The boundaries depend on the positions alone, so results stay reproducible.
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
    // the grid covers every slot once: a destination lies below its extent
    const int dest = (int)PN_IDX(hist[b * kSortBins + d] + cnt[w][d] + rank,
                                 (int64_t)gridDim.x * kSortBlock, 20);
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
    const int64_t slot = PN_IDX(perm[k], (int64_t)gridDim.x * kPackTile, 21);
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

constexpr int kOpsFar = 40, kOpsNear = 46;     // FP32-pipe operations per pair of the two bodies
constexpr int kRowThreads = 256;
constexpr int kScanThreads = 1024;

// Global target-block row r (slots [r TI, (r + 1) TI)) of the packed kernel
// with NP target pairs per thread: unit costs, their exclusive prefix within
// the row (prefix[u]) and the row total (rowsum[r]).
template <int NP>
__global__ void __launch_bounds__(kRowThreads)
k_unit_cost(const Clu *__restrict__ clu, const int *__restrict__ blk_clu,
            const float4 *__restrict__ box, float theta, int *__restrict__ prefix,
            int *__restrict__ rowsum)
{
    constexpr int TI = 2 * NP * kMixThreads, NW = kMixThreads / 32, WG = 64 * NP;
    __shared__ float4 wlo[NW], whi[NW];
    __shared__ int part[kRowThreads];
    const int64_t r = blockIdx.x;
    const Clu C = clu[cluster_of_block(blk_clu, r * TI / kGlueThreads)];
    const int64_t ntiles = C.ns_pad / kPackTile;
    const int64_t u0 = C.unit0 + (r * TI - C.slot0) / TI * ntiles;
    if (threadIdx.x < NW) {             // each warp's target box (union of its tiles' boxes)
        const float4 *bb = box + 2 * ((r * TI + WG * threadIdx.x) / kPackTile);
        float4 lo = bb[0], hi = bb[1];
        for (int q = 1; q < WG / kPackTile; ++q) {
            const float4 l = bb[2 * q], h = bb[2 * q + 1];
            lo = make_float4(fminf(lo.x, l.x), fminf(lo.y, l.y), fminf(lo.z, l.z), 0.0f);
            hi = make_float4(fmaxf(hi.x, h.x), fmaxf(hi.y, h.y), fmaxf(hi.z, h.z), fmaxf(hi.w, h.w));
        }
        wlo[threadIdx.x] = lo;
        whi[threadIdx.x] = hi;
    }
    __syncthreads();
    // thread k: tiles [k ch, (k + 1) ch) of the row
    const int64_t ch = (ntiles + kRowThreads - 1) / kRowThreads;
    const int64_t q0 = threadIdx.x * ch, q1 = q0 + ch < ntiles ? q0 + ch : ntiles;
    auto cost = [&](int64_t q) {
        const int64_t j0 = C.slot0 + q * kPackTile;
        if (j0 < r * TI + TI && r * TI < j0 + kPackTile)
            return kOpsNear;            // self pairs: full separation
        const float4 l = box[2 * (j0 / kPackTile)], h = box[2 * (j0 / kPackTile) + 1];
        for (int g = 0; g < NW; ++g) {
            const float4 bl = wlo[g], bh = whi[g];
            const float gx = fmaxf(0.0f, fmaxf(l.x - bh.x, bl.x - h.x));
            const float gy = fmaxf(0.0f, fmaxf(l.y - bh.y, bl.y - h.y));
            const float gz = fmaxf(0.0f, fmaxf(l.z - bh.z, bl.z - h.z));
            const float lim = theta * (bh.w + h.w);
            if (!(gx * gx + gy * gy + gz * gz >= lim * lim))
                return kOpsNear;
        }
        return kOpsFar;
    };
    int s = 0;
    for (int64_t q = q0; q < q1; ++q)
        s += cost(q);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < kRowThreads; ++k) {
            const int c = part[k];
            part[k] = run;
            run += c;
        }
        rowsum[r] = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int64_t q = q0; q < q1; ++q) {
        prefix[u0 + q] = run;
        run += cost(q);
    }
}

// Exclusive prefix of the row totals (one block): rowbase[r], rowbase[R] = total.
__global__ void __launch_bounds__(kScanThreads)
k_row_scan(int64_t R, const int *__restrict__ rowsum, int64_t *__restrict__ rowbase)
{
    __shared__ int64_t part[kScanThreads];
    const int64_t ch = (R + kScanThreads - 1) / kScanThreads;
    const int64_t r0 = threadIdx.x * ch, r1 = r0 + ch < R ? r0 + ch : R;
    int64_t s = 0;
    for (int64_t r = r0; r < r1; ++r)
        s += rowsum[r];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int k = 0; k < kScanThreads; ++k) {
            const int64_t c = part[k];
            part[k] = run;
            run += c;
        }
        rowbase[R] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t r = r0; r < r1; ++r) {
        rowbase[r] = run;
        run += rowsum[r];
    }
}

// Worker boundaries wb[0..G]: wb[w] = first unit u with cost prefix
// rowbase[row(u)] + prefix[u] >= w total / G (wb[G] = T).
template <int NP>
__global__ void __launch_bounds__(kGlueThreads)
k_worker_bounds(const Clu *__restrict__ clu, int nclu, int64_t T, int64_t G, int64_t R,
                const int *__restrict__ prefix, const int64_t *__restrict__ rowbase,
                int64_t *__restrict__ wb)
{
    constexpr int TI = 2 * NP * kMixThreads;
    const int64_t w = (int64_t)blockIdx.x * kGlueThreads + threadIdx.x;
    if (w > G)
        return;
    const int64_t total = rowbase[R];
    const int64_t want = w * total / G;       // total < 2^40, w <= 2^20
    auto cum = [&](int64_t u) -> int64_t {
        if (u >= T)
            return total;
        const Clu C = clu[cluster_of_unit(clu, nclu, u)];
        const int64_t ntiles = C.ns_pad / kPackTile;
        return rowbase[C.slot0 / TI + (u - C.unit0) / ntiles] + prefix[u];
    };
    int64_t lo = 0, hi = T;                   // first u in [0, T] with cum(u) >= want
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cum(mid) >= want)
            hi = mid;
        else
            lo = mid + 1;
    }
    wb[w] = w == G ? T : lo;
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

size_t balance_buffer_bytes(int64_t S, int64_t units, int64_t G)
{
    const int64_t R = S / kGlueThreads;       // target-block rows, at most (TI >= 256)
    return sizeof(int64_t) * (size_t)(R + 1 + G + 1) + sizeof(int) * (size_t)(R + units);
}

cudaError_t launch_worker_balance(pn_ctx *c, int NP, const int64_t **wb_out)
{
    const int64_t S = c->S, TI = 2 * NP * kMixThreads, R = S / TI;
    const int64_t T = c->fused_units, G = c->fused_G;
    const int64_t Rmax = S / kGlueThreads;
    int64_t *rowbase = reinterpret_cast<int64_t *>(c->bal);
    int64_t *wb = rowbase + Rmax + 1;
    int *rowsum = reinterpret_cast<int *>(wb + c->bal_G + 1);
    int *prefix = rowsum + Rmax;
    const int *bc = c->nclu > 1 ? c->blk_clu : nullptr;
    const Order o = order_of(c);
    if (NP == 2)
        k_unit_cost<2><<<(unsigned)R, kRowThreads, 0, c->stream>>>(c->d_clu, bc, o.box, c->far_theta,
                                                                   prefix, rowsum);
    else
        k_unit_cost<1><<<(unsigned)R, kRowThreads, 0, c->stream>>>(c->d_clu, bc, o.box, c->far_theta,
                                                                   prefix, rowsum);
    k_row_scan<<<1, kScanThreads, 0, c->stream>>>(R, rowsum, rowbase);
    const unsigned nb = (unsigned)((G + 1 + kGlueThreads - 1) / kGlueThreads);
    if (NP == 2)
        k_worker_bounds<2><<<nb, kGlueThreads, 0, c->stream>>>(c->d_clu, c->nclu, T, G, R, prefix,
                                                               rowbase, wb);
    else
        k_worker_bounds<1><<<nb, kGlueThreads, 0, c->stream>>>(c->d_clu, c->nclu, T, G, R, prefix,
                                                               rowbase, wb);
    c->launches += 3;
    *wb_out = wb;
    return cudaGetLastError();
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

PN_DEBUG_ACCESSOR(debug_take_order)

}  // namespace pn
