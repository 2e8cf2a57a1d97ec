// bsd_noalloc.cu -- bsd_decode_noalloc: decoding without any device allocation.
//
// The beam workspace of bsd_decode (seed store, beam window, work lists,
// counters) is carved here out of one file-scope static device array instead
// of the decoder's cudaMalloc'd workspace.  The kernels are the same ones
// bsd_decode launches; only the scratch they are pointed at differs.  The
// launches are issued one by one (the decoder's CUDA graph is bound to its own
// workspace), reading each chunk's number of active shots back through a
// static host word.
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

std::mutex g_mu;                 // serialises the address lookup and the host readback word
void* g_addr[kMaxDevices] = {};
int g_nactive = 0;

// device address of the static array on the current device (looked up once)
int scratch_address(int device, void** out)
{
    if (device < 0 || device >= kMaxDevices) return BSD_ERR_UNSUPPORTED;
    if (!g_addr[device]) {
        void* ptr = nullptr;
        if (CUDA_FAILED(cudaGetSymbolAddress(&ptr, g_bsd_scratch)) || ptr == nullptr) {
            cudaGetLastError();
            return BSD_ERR_CUDA;
        }
        g_addr[device] = ptr;
    }
    *out = g_addr[device];
    return BSD_OK;
}

// seed-store and window sizes that fit the array: the largest window with a
// seed store of four times its size, or a window of one active shot
bool fit(const DevGraph& g, const DecCfg& cfg, long long* S, long long* A)
{
    if (work_layout(g, cfg, 1, 1, nullptr, nullptr) > kScratchBytes) return false;
    long long lo = 1, hi = 2;
    while (hi < (1ll << 20) && work_layout(g, cfg, 4 * hi, hi, nullptr, nullptr) <= kScratchBytes) hi *= 2;
    while (hi - lo > 1) {
        const long long mid = (lo + hi) / 2;
        if (work_layout(g, cfg, 4 * mid, mid, nullptr, nullptr) <= kScratchBytes) lo = mid; else hi = mid;
    }
    *A = lo;
    *S = work_layout(g, cfg, 4 * lo, lo, nullptr, nullptr) <= kScratchBytes ? 4 * lo : lo;
    return true;
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
    if (!dec || B < 0) return BSD_ERR_INVALID_ARG;
    const int vrc = decoder_view(dec, &g, &cfg, &ls, &device);
    if (vrc != BSD_OK) return vrc;
    if (B == 0) return BSD_OK;
    if (!d_syndromes || !d_corrections || !d_status || (g->K > 0 && !d_obs_flips)) return BSD_ERR_INVALID_ARG;
    long long S, A;
    if (!fit(*g, *cfg, &S, &A)) return BSD_ERR_SCRATCH;

    std::lock_guard<std::mutex> lk(g_mu);
    int prev = -1;
    if (CUDA_FAILED(cudaGetDevice(&prev))) prev = -1;
    if (CUDA_FAILED(cudaSetDevice(device))) return BSD_ERR_CUDA;
    void* base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc == BSD_OK) {
        Work w{};
        work_layout(*g, *cfg, S, A, (char*)base, &w);
        cudaStream_t s = (cudaStream_t)cuda_stream;
        Outputs o{d_corrections, g->K > 0 ? d_obs_flips : nullptr, d_status, d_iters};
        // the launch statistics in the array's head start at zero; each chunk
        // resets its own counters and run descriptor (k_begin_chunk), and
        // everything else is written before it is read
        if (CUDA_FAILED(cudaMemsetAsync(w.stats, 0, kStats * sizeof(unsigned long long), s))) rc = BSD_ERR_CUDA;
        for (long long b0 = 0; b0 < B && rc == BSD_OK; b0 += S) {
            const long long n = (B - b0) < S ? (B - b0) : S;
            if (launch_chunk(*g, *cfg, w, *ls, d_syndromes, b0, n, o, s, nullptr, nullptr, &g_nactive) != 0)
                rc = BSD_ERR_CUDA;
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
