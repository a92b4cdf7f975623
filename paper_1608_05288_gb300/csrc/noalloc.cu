// util_bucket_noalloc: the single-bucket UTIL computation of util_bucket,
// for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a bucket:
// real-time or embedded loops that forbid allocation after start-up (an
// allocation can block, fail or fragment memory at a time nobody chose), and
// processes whose device memory is entirely owned by another allocator (a
// framework's caching allocator, a pre-reserved pool), where a cudaMalloc
// from this library would compete for memory it does not manage.
// util_bucket keeps a per-device scratch buffer that it grows with
// cudaMalloc; this entry point instead uses a fixed scratch array that is part
// of the library image (kNoAllocScratchBytes per device, held from the moment
// the library is loaded until the process exits) and calls no allocation
// routine at all.  The caller still owns and passes the input and output
// tables.  util_bucket_scratch_bytes reports, on the host alone, how much
// scratch a bucket needs, so a caller can tell beforehand whether the fixed
// array holds it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gpube_internal.h"

using namespace gpube;

namespace {

// Scratch of the no-allocation entry point: the bucket's offset tables, its
// descriptors and its work-queue counter and status word.  Every call shares
// it and it keeps the last call's contents; the counter and status are
// cleared by each call before its launch.
constexpr size_t kNoAllocScratchBytes = 4u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch, one per device, looked up by the first
// call made with that device current.  The address belongs to the device's
// context of that moment: after cudaDeviceReset (or any other end of the
// primary context) the module is loaded again and the cached address is no
// longer valid, so such a process must not call util_bucket_noalloc again.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

int scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return set_error(GPUBE_ENODEV, "device %d out of range", dev);
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return GPUBE_OK;
}

// The single-bucket problem of util_bucket (separator position j is variable
// j; the eliminated variable is m and goes first) planned and laid out on the
// host: no CUDA call.  The input pointers are not looked at (in_tables may be
// NULL for a size query).
int plan_bucket(int32_t cost_type, int32_t top_k, int32_t m, const int32_t *sep_dom, int32_t d, int32_t n_in,
                const void *const *in_tables, const int32_t *in_pos_off, const int32_t *in_pos, void *out,
                uint8_t *arg, wcsp &w, util_state &s)
{
    if (cost_type != WCSP_INT32_SAT && cost_type != WCSP_FP32_LOG)
        return set_error(GPUBE_EINVAL, "unknown cost type");
    if (cost_type == WCSP_INT32_SAT && top_k < 1) return set_error(GPUBE_EINVAL, "top_k must be >= 1");
    if (m < 0 || d < 1 || d > 255 || n_in < 1 || (m > 0 && !sep_dom) || !in_pos_off)
        return set_error(GPUBE_EINVAL, "bad argument");
    w.n = m + 1;
    w.cost_type = cost_type;
    w.top_k = static_cast<uint32_t>(cost_type == WCSP_INT32_SAT ? top_k : 1);
    w.dom.resize(m + 1);
    for (int j = 0; j < m; ++j) {
        if (sep_dom[j] < 1 || sep_dom[j] > 255) return set_error(GPUBE_EINVAL, "bad domain at %d", j);
        w.dom[j] = sep_dom[j];
    }
    w.dom[m] = d;
    s.w = &w;
    s.ktype = cost_type == WCSP_FP32_LOG ? kKTypeFloat : kKTypeInt;
    Plan &P = s.plan;
    P.kind = GPUBE_KIND_BE;
    P.order.resize(m + 1);
    P.pos.resize(m + 1);
    P.order[0] = m;
    for (int j = 0; j < m; ++j) P.order[1 + j] = m - 1 - j;
    for (int t = 0; t <= m; ++t) P.pos[P.order[t]] = t;
    Task T;
    T.var = m;
    T.d = d;
    T.rows = 1;
    for (int j = 0; j < m; ++j) {
        T.sep.push_back(j);
        T.rows *= sep_dom[j];
        if (T.rows > INT32_MAX) return set_error(GPUBE_ENOMEM, "output of more than 2^31 entries");
    }
    for (int i = 0; i < n_in; ++i) {
        Func f;
        const int a = in_pos_off[i], b = in_pos_off[i + 1];
        if (b < a || (b > a && !in_pos)) return set_error(GPUBE_EINVAL, "bad in_pos_off");
        int prev = -1;
        for (int k = a; k < b; ++k) {
            if (in_pos[k] <= prev || in_pos[k] >= m) return set_error(GPUBE_EINVAL, "in_pos must ascend in [0, m)");
            prev = in_pos[k];
            f.scope.push_back(in_pos[k]);
            f.size *= sep_dom[in_pos[k]];
        }
        f.scope.push_back(m);
        f.size *= d;
        if (in_tables) {
            if (!in_tables[i] || reinterpret_cast<uintptr_t>(in_tables[i]) % 16)
                return set_error(GPUBE_EINVAL, "input %d is NULL or not 16-byte aligned", i);
            f.ext = in_tables[i];
        } else {
            f.ext = &w;  // any non-null marker: the table is the caller's, outside the scratch
        }
        P.funcs.push_back(f);
        T.inputs.push_back(i);
    }
    T.ext_out = out ? out : static_cast<void *>(&w);  // the output is the caller's, outside the scratch
    T.ext_arg = arg ? arg : reinterpret_cast<uint8_t *>(&w);
    P.tasks.push_back(T);
    Func o;
    o.scope = P.tasks[0].sep;
    o.size = P.tasks[0].rows;
    o.task = 0;
    P.funcs.push_back(o);
    w.nf = n_in;
    P.n_levels = 1;
    P.level_order = {0};
    P.level_off = {0, 1};
    shape_tasks(w, P);
    gpube_layout(&s);
    return GPUBE_OK;
}

}  // namespace

extern "C" int util_bucket_scratch_bytes(int32_t m, const int32_t *sep_dom, int32_t d, int32_t n_in,
                                         const int32_t *in_pos_off, const int32_t *in_pos, size_t *bytes,
                                         size_t *noalloc_limit)
{
    if (!bytes) return set_error(GPUBE_EINVAL, "bytes is NULL");
    wcsp w;
    util_state s;
    int rc = plan_bucket(WCSP_INT32_SAT, 1, m, sep_dom, d, n_in, nullptr, in_pos_off, in_pos, nullptr, nullptr, w,
                         s);
    if (rc) return rc;
    *bytes = s.arena_bytes;
    if (noalloc_limit) *noalloc_limit = kNoAllocScratchBytes;
    return GPUBE_OK;
}

extern "C" int util_bucket_noalloc(int32_t cost_type, int32_t top_k, int32_t m, const int32_t *sep_dom,
                                   int32_t d, int32_t n_in, const void *const *in_tables,
                                   const int32_t *in_pos_off, const int32_t *in_pos, void *out, uint8_t *arg,
                                   void *stream)
{
    if (!in_tables || !out || !arg) return set_error(GPUBE_EINVAL, "bad argument");
    wcsp w;
    util_state s;
    // planning and the size check come first and make no CUDA call: a bucket
    // the fixed scratch cannot hold is rejected before anything is launched
    int rc = plan_bucket(cost_type, top_k, m, sep_dom, d, n_in, in_tables, in_pos_off, in_pos, out, arg, w, s);
    if (rc) return rc;
    if (s.arena_bytes > kNoAllocScratchBytes)
        return set_error(GPUBE_ENOMEM,
                         "util_bucket_noalloc: this bucket needs %zu bytes of scratch, the fixed scratch holds %zu "
                         "(use util_bucket)",
                         s.arena_bytes, kNoAllocScratchBytes);
    s.launch_mode = kLaunchPerTask;
    s.use_graph = false;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    s.device = dev;
    e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
    s.stream = static_cast<cudaStream_t>(stream);
    e = kernels_init_device();
    if (e != cudaSuccess) return cuda_error(e, "kernel attributes");
    rc = scratch_address(dev, &s.base);
    if (rc) return rc;
    rc = gpube_build_descriptors(&s);
    if (rc) return rc;
    const DescLayout &D = s.dl;
    const Plan &P = s.plan;
    e = cudaMemcpyAsync(s.base + s.desc_off, s.host_blob.data(), s.host_blob.size(), cudaMemcpyHostToDevice,
                        s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.base + s.status_off, 0, 8, s.stream);  // status starts at zero
    if (e == cudaSuccess)
        e = launch_expand(reinterpret_cast<const ExpandDev *>(s.base + D.expand),
                          reinterpret_cast<const int64_t *>(s.base + D.exp_prefix), 1,
                          P.tasks[0].G + 1 + P.tasks[0].P_lo, reinterpret_cast<const int32_t *>(s.base + D.pool),
                          s.num_sms, s.stream);
    if (e != cudaSuccess) return cuda_error(e, "util_bucket_noalloc upload");
    return gpube_enqueue_util(&s, s.stream);  // clears the work-queue counter, then launches
}
