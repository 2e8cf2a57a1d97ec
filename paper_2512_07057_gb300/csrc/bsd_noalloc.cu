// bsd_noalloc.cu -- bsd_decode_noalloc: decoding without any device allocation.
//
// The beam workspace of bsd_decode (child slots, per-shot bookkeeping, work
// lists, counters) is carved here out of one file-scope static device array
// instead of the decoder's cudaMalloc'd workspace.  The kernels are the same
// ones bsd_decode launches; only the scratch they are pointed at differs.
//
// Host code must not pass g_bsd_scratch itself to a kernel: in host code that
// name is a host-side stand-in, not a device address.  The device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call that decodes on it.
#include <cuda_runtime.h>

#include <mutex>

#include "bsd.h"
#include "bsd_internal.cuh"

namespace bsd {
int decoder_view(const bsd_decoder* dec, const DevGraph** g, const DecCfg** cfg, const LaunchShape** ls,
                 int* device);
}

using namespace bsd;

namespace {

constexpr size_t kScratchBytes = BSD_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bsd_scratch[kScratchBytes];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// byte offsets of the workspace arrays for a chunk of C shots (same arrays as
// the decoder's own workspace); returns the total size
size_t layout(const DevGraph& g, const DecCfg& cfg, long long C, char* base, Work* w)
{
    const size_t W2 = 2 * (size_t)cfg.w;
    const size_t SB = (size_t)g.WM + 3 * (size_t)g.WN;
    const size_t NR = (size_t)cfg.num_results;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += a256(bytes > 0 ? bytes : 1);
        return base + o;
    };
    const size_t ctr_bytes = a256(sizeof(Counters) + sizeof(int) * 3 * (size_t)(cfg.max_rounds + 2));
    char* ctr = take(ctr_bytes);
    char* stats = take(2 * sizeof(unsigned long long));
    if (w) {
        w->ctr = reinterpret_cast<Counters*>(ctr);
        w->round_ctr = reinterpret_cast<int*>(ctr + sizeof(Counters));
        w->stats = reinterpret_cast<unsigned long long*>(stats);
        w->C = C;
        w->SB = (int)SB;
    }
    char* p;
    p = take(sizeof(float) * 2 * C * W2 * (size_t)g.Epad);      if (w) w->slotE = (float*)p;
    p = take(sizeof(uint32_t) * 2 * C * W2 * SB);               if (w) w->slotBits = (uint32_t*)p;
    p = take(sizeof(SlotMeta) * 2 * C * W2);                    if (w) w->slotMeta = (SlotMeta*)p;
    p = take(sizeof(int) * C);                                  if (w) w->shot_of = (int*)p;
    p = take(sizeof(int) * C);                                  if (w) w->set_size = (int*)p;
    p = take(sizeof(int) * C);                                  if (w) w->done = (int*)p;
    p = take((size_t)C * cfg.w);                                if (w) w->set_idx = (uint8_t*)p;
    p = take(sizeof(unsigned long long) * C);                   if (w) w->iters_acc = (unsigned long long*)p;
    p = take(sizeof(uint32_t) * C * NR * (size_t)g.WN);         if (w) w->res_bits = (uint32_t*)p;
    p = take(sizeof(long long) * C * NR);                       if (w) w->res_w = (long long*)p;
    p = take(sizeof(int) * C * NR);                             if (w) w->res_origin = (int*)p;
    p = take(sizeof(int) * C);                                  if (w) w->res_n = (int*)p;
    p = take(sizeof(int2) * 2 * C * W2);                        if (w) w->items = (int2*)p;
    return off;
}

// device address of the static array on the current device (looked up once)
int scratch_address(int device, void** out)
{
    if (device < 0 || device >= kMaxDevices) return BSD_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[device]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_bsd_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return BSD_ERR_CUDA;
        }
        g_addr[device] = ptr;
    }
    *out = g_addr[device];
    return BSD_OK;
}

}  // namespace

extern "C" int bsd_decode_noalloc(const bsd_decoder* dec, const uint32_t* d_syndromes, int64_t B,
                                  uint32_t* d_corrections, uint32_t* d_obs_flips, uint32_t* d_status,
                                  uint32_t* d_iters, void* cuda_stream)
{
    const DevGraph* g;
    const DecCfg* cfg;
    const LaunchShape* ls;
    int device;
    if (!dec || B < 0 || decoder_view(dec, &g, &cfg, &ls, &device) != BSD_OK) return BSD_ERR_INVALID_ARG;
    if (B == 0) return BSD_OK;
    if (!d_syndromes || !d_corrections || !d_status || (g->K > 0 && !d_obs_flips)) return BSD_ERR_INVALID_ARG;
    // the largest chunk whose workspace fits the array; one shot must fit
    if (layout(*g, *cfg, 1, nullptr, nullptr) > kScratchBytes) return BSD_ERR_SCRATCH;
    long long lo = 1, hi = 1;
    while (hi < (1ll << 22) && layout(*g, *cfg, hi * 2, nullptr, nullptr) <= kScratchBytes) hi *= 2;
    lo = hi;
    hi = hi * 2;
    while (hi - lo > 1) {
        const long long mid = (lo + hi) / 2;
        if (layout(*g, *cfg, mid, nullptr, nullptr) <= kScratchBytes) lo = mid; else hi = mid;
    }
    const long long C = lo;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(device) != cudaSuccess) return BSD_ERR_CUDA;
    int rc = BSD_OK;
    void* base = nullptr;
    rc = scratch_address(device, &base);
    if (rc == BSD_OK) {
        Work w{};
        const size_t ctr_bytes = a256(sizeof(Counters) + sizeof(int) * 3 * (size_t)(cfg->max_rounds + 2));
        layout(*g, *cfg, C, (char*)base, &w);
        cudaStream_t s = (cudaStream_t)cuda_stream;
        Outputs o{d_corrections, g->K > 0 ? d_obs_flips : nullptr, d_status, d_iters};
        for (long long b0 = 0; b0 < B && rc == BSD_OK; b0 += C) {
            const long long n = (B - b0) < C ? (B - b0) : C;
            // per-chunk counters and the iteration statistics start at zero;
            // everything else is written before it is read
            if (cudaMemsetAsync(base, 0, ctr_bytes + a256(2 * sizeof(unsigned long long)), s) != cudaSuccess ||
                launch_chunk(*g, *cfg, w, *ls, d_syndromes, b0, n, o, s, nullptr) != 0)
                rc = BSD_ERR_CUDA;
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
