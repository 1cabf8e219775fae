// mdx_simulate_strings_noalloc: a forward run of strings and membranes that
// allocates no device memory.
//
// Who needs it: callers that must not call cudaMalloc.  A real-time audio
// callback cannot afford it (cudaMalloc can block for milliseconds and
// synchronises the device, so the audio deadline would be missed), and a
// plug-in running inside a host application that owns every device buffer is
// not allowed to allocate behind the host's back.  Such callers pass their
// own input and output buffers; everything else the run needs lives in one
// fixed block of device memory that belongs to this library.
//
// The block is the file-scope array g_noalloc_scratch below.  Every GPU that
// loads the library keeps it until the process exits.  Host code cannot use
// the array's name as a device address (it is a host-side handle), so on the
// first call on each device, with that device current, the device address is
// looked up once with cudaGetSymbolAddress and cached.  Because that set-up
// runs on the first call, the first call on a device should happen before any
// stream capture.
//
// The per-call table (instance descriptions and FP32 coefficients, computed
// on the host) reaches the block inside the parameters of small copy kernels,
// at most 31 KB per launch: no host buffer is read after the call returns and
// no pageable host-to-device copy is issued.
//
// All calls share the block and it keeps whatever the last call wrote.
// Nothing in it has to start at zero: each call writes every word it later
// reads (instance table, coefficients, state).  Calls whose work overlaps on
// the GPU (for example on two streams) race on the block and corrupt each
// other; serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/mdx.h"
#include "mdx_internal.h"
#include "mdx_scheme.cuh"

using namespace mdx;

namespace {

constexpr size_t kNoAllocBytes = size_t(1) << 20;   // 1 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

int noalloc_fail(int code, const char *msg) { return set_last_error(code, msg); }

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// The size limit stated in include/mdx.h counts 120 bytes per instance
// descriptor.
static_assert(sizeof(InstDesc) == 120, "update the no-allocation size limit in mdx.h");

// One piece of the host table, carried by value in the kernel's parameters
// (kernel parameters may hold up to 32 764 bytes).
constexpr int kUploadWords = 7936;
struct UploadChunk {
    unsigned *dst;
    int n;
    unsigned w[kUploadWords];
};

__global__ void noalloc_upload_kernel(const __grid_constant__ UploadChunk c) {
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) c.dst[i] = c.w[i];
}

}  // namespace

// Largest total mode count the fixed block can hold for n_inst instances.
static long noalloc_max_modes(int n_inst) {
    if (n_inst < 1) return 0;
    const size_t head = align16((size_t)n_inst * sizeof(InstDesc)) + align16((size_t)n_inst * sizeof(int));
    if (head >= kNoAllocBytes) return 0;
    // 8 coefficient arrays + 4 state arrays, each 16-byte aligned
    return (long)((kNoAllocBytes - head - 12 * 16) / (12 * sizeof(float)));
}

extern "C" int mdx_simulate_strings_noalloc(const mdx_instance *inst, int n_inst, const float *exc,
                                            const double *q0, const double *qm1, int steps,
                                            float *audio, double *q_end, double *qm1_end,
                                            int *status, void *stream) {
    if (!inst || n_inst < 1) return noalloc_fail(MDX_ERR_ARG, "need at least one instance");
    if (steps < 0) return noalloc_fail(MDX_ERR_ARG, "steps must be >= 0");
    long long TM = 0;
    int max_n = 1;
    for (int i = 0; i < n_inst; ++i) {
        const mdx_instance &I = inst[i];
        if (I.kind != MDX_KIND_TENSION)
            return noalloc_fail(MDX_ERR_ARG, "only strings and membranes (MDX_KIND_TENSION)");
        if (I.n_phi < 1 || I.n_phi > MDX_MAX_PHI)
            return noalloc_fail(MDX_ERR_UNSUPPORTED, "n_phi outside [1, MDX_MAX_PHI]");
        if (!I.omega2 || !I.gamma || !I.b || !I.c || !I.lambda)
            return noalloc_fail(MDX_ERR_ARG, "omega2, gamma, b, c and lambda are required");
        if (!(I.dt > 0.0) || !std::isfinite(I.dt) || !std::isfinite(I.tau) || I.tau < 0.0)
            return noalloc_fail(MDX_ERR_ARG, "dt must be > 0 and tau finite and >= 0");
        for (int m = 0; m < I.n_phi; ++m) {
            if (!std::isfinite(I.omega2[m]) || !std::isfinite(I.gamma[m]) ||
                !std::isfinite(I.b[m]) || !std::isfinite(I.c[m]) || !std::isfinite(I.lambda[m]))
                return noalloc_fail(MDX_ERR_NONFINITE, "non-finite coefficient");
            if (!(I.omega2[m] > 0.0) || I.lambda[m] < 0.0)
                return noalloc_fail(MDX_ERR_ARG, "omega2 must be > 0 and lambda >= 0");
            if (I.gamma[m] < 0.0 || std::sqrt(I.omega2[m]) * I.dt >= 2.0)
                return noalloc_fail(MDX_ERR_UNSTABLE, "gamma < 0 or omega*dt >= 2");
        }
        TM += I.n_phi;
        max_n = I.n_phi > max_n ? I.n_phi : max_n;
    }
    if (TM > noalloc_max_modes(n_inst))
        return noalloc_fail(MDX_ERR_UNSUPPORTED,
                            "total modes exceed the fixed 1 MiB scratch block of the "
                            "no-allocation entry point (at most (1048576 - align16(120 n) - "
                            "align16(4 n) - 192) / 48 for n instances)");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(MDX_ERR_CUDA, "no usable current device");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *addr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess || !addr)
                return noalloc_fail(MDX_ERR_CUDA, "cudaGetSymbolAddress of the scratch block failed");
            g_scratch_addr[dev] = addr;
        }
        base = g_scratch_addr[dev];
    }

    // Host image of the instance table, instance list and coefficients
    // (host memory only), copied into the fixed block.
    const size_t off_list = align16(n_inst * sizeof(InstDesc));
    const size_t off_coef = off_list + align16(n_inst * sizeof(int));
    const size_t coef_stride = align16(TM * sizeof(float));
    const size_t off_state = off_coef + 8 * coef_stride;
    std::vector<unsigned char> img(off_state, 0);
    InstDesc *desc = reinterpret_cast<InstDesc *>(img.data());
    int *list = reinterpret_cast<int *>(img.data() + off_list);
    float *cf = reinterpret_cast<float *>(img.data() + off_coef);
    const size_t cs = coef_stride / sizeof(float);
    long long mo = 0;
    for (int i = 0; i < n_inst; ++i) {
        const mdx_instance &I = inst[i];
        InstDesc d{};
        d.kind = MDX_KIND_TENSION;
        d.N = I.n_phi;
        d.Npad = (I.n_phi + 3) & ~3;
        d.mode_off = mo;
        d.taup = (float)I.tau;
        desc[i] = d;
        list[i] = i;
        const double T = I.dt;
        for (int m = 0; m < I.n_phi; ++m) {
            // the same FP32 coefficients as a plan of scheme MDX_SCHEME_SV
            const ModeF32 k = mode_f32(MDX_SCHEME_SV, I.omega2[m], I.gamma[m], T);
            cf[0 * cs + mo + m] = k.eps;
            cf[1 * cs + mo + m] = k.rho_hi;
            cf[2 * cs + mo + m] = k.r;
            cf[3 * cs + mo + m] = (float)I.b[m];
            cf[4 * cs + mo + m] = (float)I.c[m];
            cf[5 * cs + mo + m] = (float)I.lambda[m];
            cf[6 * cs + mo + m] = k.rho_lo;
            cf[7 * cs + mo + m] = (float)(I.c[m] - (double)(float)I.c[m]);
        }
        mo += I.n_phi;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *b = static_cast<unsigned char *>(base);
    {
        // the table, in kernel-parameter pieces (its size is a multiple of 16 bytes)
        static thread_local UploadChunk chunk;
        const unsigned *words = reinterpret_cast<const unsigned *>(img.data());
        const size_t n_words = img.size() / sizeof(unsigned);
        for (size_t w0 = 0; w0 < n_words; w0 += kUploadWords) {
            const int n = (int)std::min<size_t>(kUploadWords, n_words - w0);
            chunk.dst = reinterpret_cast<unsigned *>(b) + w0;
            chunk.n = n;
            std::memcpy(chunk.w, words + w0, (size_t)n * sizeof(unsigned));
            noalloc_upload_kernel<<<1, 256, 0, s>>>(chunk);
            if (cudaGetLastError() != cudaSuccess)
                return noalloc_fail(MDX_ERR_CUDA, "copy into the scratch block failed");
        }
    }
    if (status && cudaMemsetAsync(status, 0, n_inst * sizeof(int), s) != cudaSuccess)
        return noalloc_fail(MDX_ERR_CUDA, "clearing status failed");
    const float *dcf = reinterpret_cast<const float *>(b + off_coef);
    float *state = reinterpret_cast<float *>(b + off_state);
    AuxInit a{q0, qm1, state, TM};
    if (launch_init_state(a, s) != cudaSuccess)
        return noalloc_fail(MDX_ERR_CUDA, "state initialisation launch failed");
    if (steps > 0) {
        TensionParams T{};
        T.inst = reinterpret_cast<const InstDesc *>(b);
        T.list = reinterpret_cast<const int *>(b + off_list);
        T.n_list = n_inst;
        T.coef.eps = dcf;
        T.coef.rw2 = dcf + cs;
        T.coef.r = dcf + 2 * cs;
        T.coef.b = dcf + 3 * cs;
        T.coef.c = dcf + 4 * cs;
        T.coef.lam = dcf + 5 * cs;
        T.coef.rw2lo = dcf + 6 * cs;
        T.coef.clo = dcf + 7 * cs;
        T.steps = steps;
        T.n_begin = 0;
        T.total_steps = steps;
        T.mode = MODE_FORWARD;
        T.exc = exc;
        T.audio = audio;
        T.state_io = state;
        T.ckpt_K = 1 << 30;
        T.total_modes = TM;
        T.status = status;
        if (launch_tension(T, max_n, s) != cudaSuccess)
            return noalloc_fail(MDX_ERR_CUDA, "tension kernel launch failed");
    }
    if (launch_finalize_state(state, TM, q_end, qm1_end, s) != cudaSuccess)
        return noalloc_fail(MDX_ERR_CUDA, "state finalisation launch failed");
    return MDX_OK;
}
