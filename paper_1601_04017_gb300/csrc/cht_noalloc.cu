// cht_find_noalloc: a find that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc (or cudaMallocAsync) at
// the point where they look keys up -- e.g. a process whose device memory is
// already reserved by another allocator (a framework's caching pool or a
// serving system's fixed arena), so any extra allocation could fail or
// fragment it; a latency-critical request path where an allocation or free
// might block or synchronize the device; or an embedding with a fixed memory
// budget that must know every byte the library holds in advance.  cht_find
// itself allocates only when it is given host arrays (it stages them through
// stream-ordered device buffers); this entry point stages through one fixed
// scratch array instead.
//
// The scratch is a file-scope __device__ array of kNoallocMaxKeys * 17 bytes
// (about 1.1 MiB: keys, values, result codes).  Every GPU that loads the
// library holds it until the process exits.  Host code never passes the
// array's symbol to a kernel (in host code that name is only a stand-in);
// its device address is looked up once per device with
// cudaGetSymbolAddress, on that device, during the first call there.
#include <mutex>

#include "../../include/cht.h"
#include "cht_internal.h"

namespace {

constexpr unsigned long long kNoallocMaxKeys = CHT_NOALLOC_MAX_KEYS;
constexpr unsigned long long kScratchBytes = kNoallocMaxKeys * (8 + 8 + 1);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once).
cht_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return CHT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return CHT_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return CHT_OK;
}

}  // namespace

extern "C" cht_status cht_find_noalloc(cht_handle h, const uint64_t* keys, uint64_t n, uint64_t* vals_out,
                                       uint8_t* found, cht_stream_t stream) {
    if (!h || (n > 0 && (!keys || !vals_out))) return CHT_ERR_INVALID_ARG;
    if (n > kNoallocMaxKeys) return CHT_ERR_INVALID_ARG;
    if (n == 0) return CHT_OK;
    cht::Cell* cells = nullptr;
    cht::u32 log2c = 0;
    cht::DevState* st = nullptr;
    int device = 0, group_width = 1, lane_cells = 2, ctas_per_sm = 0, full_keys = 0;
    cht::table_view(h, &cells, &log2c, &st, &device, &group_width, &lane_cells, &ctas_per_sm, &full_keys);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return CHT_ERR_CUDA;
    cht_status r = CHT_OK;
    unsigned char* base = nullptr;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the find reads the cells on s: cht_destroy (and a migration that frees
    // the cells) must order itself after it, as after every other call
    cht::table_note_stream(h, s);
    if ((r = scratch_address(device, &base)) == CHT_OK) {
        cht::u64* s_keys = reinterpret_cast<cht::u64*>(base);
        cht::u64* s_vals = s_keys + kNoallocMaxKeys;
        unsigned char* s_codes = reinterpret_cast<unsigned char*>(s_vals + kNoallocMaxKeys);
        // Nothing in the scratch must start at zero: the kernel writes a value
        // and a code for every key of the batch.
        if (cudaMemcpyAsync(s_keys, keys, n * 8, cudaMemcpyDefault, s) != cudaSuccess) {
            r = CHT_ERR_CUDA;
        } else {
            cht::OpArgs a;
            a.cells = cells;
            a.log2c = log2c;
            a.reuse = 0;  // finds never take cells
            a.full_keys = cht::u32(full_keys);
            a.keys = s_keys;
            a.vals = nullptr;
            a.vals_out = s_vals;
            a.codes = found ? s_codes : nullptr;
            a.n = n;
            a.st = st;
            if (cht::launch_op(cht::kFind, a, group_width, lane_cells, ctas_per_sm, s) != cudaSuccess ||
                cudaMemcpyAsync(vals_out, s_vals, n * 8, cudaMemcpyDefault, s) != cudaSuccess ||
                (found && cudaMemcpyAsync(found, s_codes, n, cudaMemcpyDefault, s) != cudaSuccess))
                r = CHT_ERR_CUDA;
        }
        if (r != CHT_OK) cudaGetLastError();
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return r;
}
