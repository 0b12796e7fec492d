// pn_noalloc.cu -- pn_energy_noalloc: the energy/momentum evaluation for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// owned by another allocator (a framework's caching pool that has reserved
// the GPU), code that must not allocate after start-up (real-time loops,
// library hooks with a fixed memory budget), or code running where
// allocation calls are forbidden.  pn_energy needs a context, and pn_init
// allocates; this entry point instead works in a scratch array compiled into
// the library, so it allocates nothing.
//
// The scratch is a file-scope __device__ array: every GPU that loads
// libpn holds it (kScratchBytes, about 5 MiB) until the process exits.  Its
// host-side name is only a stand-in, so its device address is looked up
// with cudaGetSymbolAddress once per device (on the first call on that
// device, with that device current) and cached; cudaDeviceReset on that
// device invalidates the cached address, so the entry point must not be
// called on a device after it was reset.  Every call shares the array;
// each call writes every scratch byte it later reads, so nothing needs
// clearing, but calls whose work overlaps on the GPU (other streams, or
// another thread) race on the array.  The one-entry cluster table is
// written by a kernel that takes it by value, so no call reads host memory
// after it returns.
#include <cmath>
#include <mutex>

#include "pn_internal.h"

namespace {

constexpr int64_t kMaxBodies = 16384;                       // PN_NOALLOC_MAX_BODIES
constexpr int64_t kPadMax = (kMaxBodies - 1 + pn::kPad - 1) / pn::kPad * pn::kPad;
constexpr int64_t kRecBytes = 2 * kPadMax * (int64_t)sizeof(double4_32a);
constexpr int64_t kPartBytes = (int64_t)pn::kEVals * kPadMax * 8;
constexpr int64_t kBlkBytes = (kPadMax / pn::kGlueThreads) * pn::kEBlockVals * 8;
constexpr int64_t kAlign = 256;
constexpr int64_t kCluOff = 0;                              // the one-entry cluster table
constexpr int64_t kRecOff = kAlign;
constexpr int64_t kPartOff = (kRecOff + kRecBytes + kAlign - 1) / kAlign * kAlign;
constexpr int64_t kBlkOff = (kPartOff + kPartBytes + kAlign - 1) / kAlign * kAlign;
constexpr int64_t kScratchBytes = (kBlkOff + kBlkBytes + kAlign - 1) / kAlign * kAlign;

// Each region holds what launch_energy_on writes for the largest padded
// star count: the energy records (2 double4 per slot), the pair sums
// (kEVals per slot) and one row of kEBlockVals per kGlueThreads-slot block.
static_assert(kPadMax % pn::kGlueThreads == 0 && kPadMax % pn::kF64Threads == 0,
              "launch_energy_on's grids cover whole blocks of the padded slots");
static_assert(kRecOff + kRecBytes <= kPartOff && kPartOff + kPartBytes <= kBlkOff &&
                  kBlkOff + kBlkBytes <= kScratchBytes,
              "scratch regions must not overlap");
static_assert((int64_t)sizeof(pn::Clu) <= kRecOff, "cluster table fits before the records");

static __device__ __align__(256) unsigned char g_energy_scratch[kScratchBytes];

// Bytes that launch_energy_on writes into each region for S padded slots
// (kept next to its launch shapes: records 2 S double4, pair sums kEVals S
// doubles, epilogue rows S / kGlueThreads of kEBlockVals doubles).
bool regions_fit(int64_t S)
{
    return 2 * S * (int64_t)sizeof(double4_32a) <= kRecBytes &&
           (int64_t)pn::kEVals * S * 8 <= kPartBytes &&
           (S / pn::kGlueThreads) * pn::kEBlockVals * 8 <= kBlkBytes;
}

__global__ void k_put_clu(pn::Clu *dst, pn::Clu src) { *dst = src; }

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices];

pn_status fail(pn_status s, const char *msg, const char *detail = "")
{
    return pn::set_error(s, "%s%s", msg, detail);
}

}  // namespace

extern "C" pn_status pn_energy_noalloc(int device, void *cuda_stream, int64_t n, double G,
                                       double c, double eps, const double *x, const double *v,
                                       const double *m, double *out)
{
    if (n < 2)
        return fail(PN_EINVAL, "pn_energy_noalloc: n must be >= 2");
    if (n > kMaxBodies)
        return fail(PN_EINVAL, "pn_energy_noalloc: n exceeds PN_NOALLOC_MAX_BODIES (16384)");
    if (!x || !v || !m || !out)
        return fail(PN_EINVAL, "pn_energy_noalloc: NULL array");
    if (!(std::isfinite(G) && G > 0.0) || !(c > 0.0) || !(std::isfinite(eps) && eps >= 0.0))
        return fail(PN_EINVAL, "pn_energy_noalloc: need G > 0, c > 0 (or INFINITY), eps >= 0");
    if (device < 0 || device >= kMaxDevices)
        return fail(PN_EINVAL, "pn_energy_noalloc: device index out of range");
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != device)
        e = cudaSetDevice(device);
    if (e != cudaSuccess)
        return fail(PN_ECUDA, "pn_energy_noalloc: cudaSetDevice: ", cudaGetErrorString(e));
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[device]) {
            e = cudaGetSymbolAddress(&g_addr[device], g_energy_scratch);
            if (e != cudaSuccess)
                g_addr[device] = nullptr;
        }
        base = g_addr[device];
    }
    if (!base) {
        if (prev >= 0 && prev != device)
            cudaSetDevice(prev);
        return fail(PN_ECUDA, "pn_energy_noalloc: cudaGetSymbolAddress: ", cudaGetErrorString(e));
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    pn::Clu clu = {};
    clu.body0 = 0;
    clu.ns = n - 1;
    clu.ns_pad = (clu.ns + pn::kPad - 1) / pn::kPad * pn::kPad;
    clu.slot0 = 0;
    clu.G = G;
    clu.inv_c2 = std::isinf(c) ? 0.0 : 1.0 / (c * c);
    clu.eps2 = eps * eps;
    clu.r_near = -1.0;
    if (!regions_fit(clu.ns_pad)) {
        if (prev >= 0 && prev != device)
            cudaSetDevice(prev);
        return fail(PN_EINVAL, "pn_energy_noalloc: padded size exceeds the scratch regions");
    }
    pn::Clu *dclu = reinterpret_cast<pn::Clu *>(b + kCluOff);
    k_put_clu<<<1, 1, 0, (cudaStream_t)cuda_stream>>>(dclu, clu);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = pn::launch_energy_on((cudaStream_t)cuda_stream, clu.ns_pad, dclu, x, v, m,
                                 reinterpret_cast<double4_32a *>(b + kRecOff),
                                 reinterpret_cast<double *>(b + kPartOff),
                                 reinterpret_cast<double *>(b + kBlkOff), out);
    if (prev >= 0 && prev != device)
        cudaSetDevice(prev);
    if (e != cudaSuccess)
        return fail(PN_ECUDA, "pn_energy_noalloc: launch: ", cudaGetErrorString(e));
    return PN_OK;
}
