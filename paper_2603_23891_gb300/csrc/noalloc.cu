// Allocation-free variant of the selection compaction.
//
// Some callers cannot call cudaMalloc: a host application that owns every
// device allocation itself (and hands a plug-in only the buffers it already
// made), code that runs while a CUDA stream is being captured into a graph,
// or a real-time loop where allocation after start-up is not allowed.  For
// them, fgs_compact_selection_noalloc() runs the same compaction kernel as the
// render path, but its scratch memory (the decoupled look-back words and the
// small frame-state block with the tile ticket, epoch and result count) lives
// in the file-scope device array below instead of context-owned memory.  The
// caller passes the input bits and the output buffers; nothing is allocated.
//
// The array holds kNoAllocScratchBytes on every GPU that loads this library,
// until the process exits.  Its name is a host-side stand-in in host code, so
// host code takes its device address with cudaGetSymbolAddress, once per
// device, with that device current.
#include "filtergs.h"
#include "fgs_internal.cuh"

#include <mutex>

namespace fgs {

namespace {

constexpr uint64_t kNoAllocMaxWords = 1ull << 26;                 // 2^31 nodes
constexpr uint64_t kNoAllocTiles = kNoAllocMaxWords / kCompactWords;  // 65536 look-back words
constexpr size_t kStateBytes = (sizeof(FrameState) + 255) / 256 * 256;
constexpr size_t kNoAllocScratchBytes = kStateBytes + kNoAllocTiles * sizeof(unsigned long long);
// The size the header documents (512 KiB of look-back words + a 256-byte
// state block); a change of FrameState must update the documentation too.
static_assert(kNoAllocScratchBytes == 524544, "documented scratch size of the no-alloc entry point");

// FrameState block first, then one 64-bit look-back word per compaction tile.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Per call: a new epoch (older look-back words then read as "not ready"), the
// ticket counter, result count and status back to zero.
__global__ void noalloc_begin_kernel(FrameState* st)
{
    st->epoch = st->epoch + 1;
    st->M = 0;
    st->tickets[kTicketCompact] = 0;
    st->status = 0;
    st->status_info = 0;
}

__global__ void noalloc_finish_kernel(const FrameState* st, uint32_t* count_out)
{
    count_out[0] = st->status == 0 ? st->M : 0xFFFFFFFFu;
}

}  // namespace
}  // namespace fgs

using namespace fgs;

extern "C" int fgs_compact_selection_noalloc(const uint32_t* selbits, uint64_t n_words,
                                             uint32_t* ids_out, uint32_t* count_out, void* stream)
{
    if (!selbits || !ids_out || !count_out || n_words == 0) return FGS_ERR_ARG;
    if (n_words > kNoAllocMaxWords) return FGS_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FGS_ERR_CUDA;
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FGS_ERR_CUDA;
            g_scratch_ptr[dev] = (unsigned char*)p;
        }
        base = g_scratch_ptr[dev];
    }
    FrameState* st = reinterpret_cast<FrameState*>(base);
    unsigned long long* lookback = reinterpret_cast<unsigned long long*>(base + kStateBytes);
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    noalloc_begin_kernel<<<1, 1, 0, s>>>(st);
    launch_compact(selbits, (uint32_t)n_words, ids_out, (uint32_t)(n_words * 32u), lookback, st,
                   sms * occ_compact(), s);
    noalloc_finish_kernel<<<1, 1, 0, s>>>(st, count_out);
    return cudaGetLastError() == cudaSuccess ? FGS_OK : FGS_ERR_CUDA;
}
