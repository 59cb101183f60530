// rtu_static.cu -- rtu_gp_source_static: the GP source step (white noise filtered
// by the square root of the power spectrum through FFTs, then the softplus map and
// the alpha power) without a caller-provided workspace, for callers that cannot
// allocate device memory.
//
// Its scratch is one file-scope __device__ array (RTU_STATIC_MAX_NSRC^2 complex
// doubles, 256 KiB) that every GPU loading this library holds until the process
// exits.  Host code cannot pass the array's name to a kernel: in host code that
// name is a host-side stand-in, not a device address.  So the host looks up the
// array's device address with cudaGetSymbolAddress (with the device current):
// at the first call on a device, and again at every later call that is not being
// captured into a CUDA graph (so a device reset between calls is picked up); a
// captured call uses the address found by the device's last uncaptured call.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "rtu.h"
#include "k_gp.cuh"

using namespace rtu;

// records the message returned by rtu_last_error() (defined with the other entry points)
rtu_status rtu_fail_internal(rtu_status code, const char* msg);

namespace {

constexpr int SMAX = RTU_STATIC_MAX_NSRC;

// the FFT buffer shared by every call of rtu_gp_source_static
static __device__ __align__(256) double2 g_gp_static_scratch[SMAX * SMAX];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

rtu_status fail_static(rtu_status code, const std::string& m) { return rtu_fail_internal(code, m.c_str()); }

// One CTA: twiddles, digit reversal and radices built in shared memory, then
// the forward FFT, the sqrt(P) filter, the inverse FFT and the softplus map, all
// in double and rounded to float at the end, like the workspace path (near f = 0
// the softplus turns an absolute error of f into a relative error of the source
// 1/s0 = 100 times larger, which rules out float transforms).
__global__ void __launch_bounds__(GP_NT) k_gp_source_static(int n, double pitch, int family, const float* lat,
                                                            const double* ps, float* out, Cx<double>* W) {
    extern __shared__ __align__(128) unsigned char smem_static[];
    Cx<double>* sm = reinterpret_cast<Cx<double>*>(smem_static);
    __shared__ Cx<double> tw_s[SMAX];
    __shared__ int rev_s[SMAX];
    __shared__ int rad_s[MAX_RADIX];
    __shared__ int nrad_s;
    if (threadIdx.x == 0) {
        int m = n, k = 0;
        while (m % 4 == 0) { rad_s[k++] = 4; m /= 4; }
        while (m % 2 == 0) { rad_s[k++] = 2; m /= 2; }
        while (m % 3 == 0) { rad_s[k++] = 3; m /= 3; }
        nrad_s = k;
    }
    __syncthreads();
    const int S = nrad_s;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double ang = -2.0 * 3.14159265358979323846 * i / n;
        tw_s[i] = Cx<double>{cos(ang), sin(ang)};
        // position p holds element rev(p): p = sum_s j_s L_{s-1} -> j_S + r_S j_{S-1} + ...
        int js[MAX_RADIX];
        int q = i;
        for (int s = 0; s < S; ++s) { js[s] = q % rad_s[s]; q /= rad_s[s]; }
        int v = 0, w = 1;
        for (int s = S - 1; s >= 0; --s) { v += js[s] * w; w *= rad_s[s]; }
        rev_s[i] = v;
    }
    __syncthreads();
    const int n2 = n * n;
    const int chunk = max(1, min(n, (int)(GP_SMEM / sizeof(Cx<double>)) / n));
    for (int i = threadIdx.x; i < n2; i += blockDim.x) W[i] = Cx<double>{(double)lat[i], 0.0};
    __syncthreads();
    fft2<double>(W, n, rad_s, S, tw_s, rev_s, sm, chunk, false);
    const int nf = n_family(family);
    double psv[4];
    for (int q = 0; q < nf; ++q) psv[q] = ps[q];
    const double kscale = 2.0 * 3.14159265358979323846 / pitch;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int ky = i / n, kx = i - ky * n;
        const double fx = fftfreq<double>(kx, n), fy = fftfreq<double>(ky, n);
        const double k = kscale * sqrt(fx * fx + fy * fy);
        double gdummy[3];
        const double sp = sqrtP_and_grad<double>(family, psv, k, gdummy);
        W[i] = Cx<double>{W[i].x * sp, W[i].y * sp};
    }
    __syncthreads();
    fft2<double>(W, n, rad_s, S, tw_s, rev_s, sm, chunk, true);
    const double alpha = ps[nf];
    const double inv_n2 = 1.0 / (double)n2;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const double f = W[i].x * inv_n2;
        out[i] = (float)exp(alpha * log_sp_s0<double>(f / 0.01));
    }
}

bool valid_size(int n) {
    if (n < 4 || n > SMAX) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

}  // namespace

extern "C" {

rtu_status rtu_gp_source_static(int32_t n_src, double src_pitch, int32_t ps_family, const float* latents,
                                const double* ps, float* source, void* stream) {
    if (!valid_size(n_src))
        return fail_static(RTU_E_ARG, "rtu_gp_source_static: n_src must be 2^a 3^b in [4, " +
                                          std::to_string(SMAX) + "] (the static scratch holds " +
                                          std::to_string(SMAX) + "^2 complex values)");
    if (ps_family < 0 || ps_family > 2) return fail_static(RTU_E_ARG, "rtu_gp_source_static: bad ps_family");
    if (!(src_pitch > 0)) return fail_static(RTU_E_ARG, "rtu_gp_source_static: src_pitch must be > 0");
    if (!latents || !ps || !source) return fail_static(RTU_E_ARG, "rtu_gp_source_static: null pointer");
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return fail_static(RTU_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    if (dev < 0 || dev >= MAX_DEVICES) return fail_static(RTU_E_ARG, "rtu_gp_source_static: device index too large");
    // the caller may be capturing this stream into a CUDA graph: then no set-up call
    // is made and the address of the device's last uncaptured call is used
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ce = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap);
    if (ce != cudaSuccess)
        return fail_static(RTU_E_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            // set-up with this device current: the static array's device address and the
            // kernel's shared-memory limit (neither allocates; both are looked up again
            // at every uncaptured call, so a device reset between calls is picked up)
            void* p = nullptr;
            ce = cudaGetSymbolAddress(&p, g_gp_static_scratch);
            if (ce != cudaSuccess)
                return fail_static(RTU_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
            ce = cudaFuncSetAttribute(k_gp_source_static, cudaFuncAttributeMaxDynamicSharedMemorySize, GP_SMEM);
            if (ce != cudaSuccess)
                return fail_static(RTU_E_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce));
            g_scratch_addr[dev] = p;
        } else if (!g_scratch_addr[dev]) {
            return fail_static(RTU_E_ARG, "rtu_gp_source_static: make a first call on this device outside "
                                          "stream capture (it looks up the scratch address)");
        }
        scratch = g_scratch_addr[dev];
    }
    k_gp_source_static<<<1, GP_NT, GP_SMEM, static_cast<cudaStream_t>(stream)>>>(
        n_src, src_pitch, ps_family, latents, ps, source, static_cast<Cx<double>*>(scratch));
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail_static(RTU_E_CUDA, std::string("launch: ") + cudaGetErrorString(ce));
    return RTU_OK;
}

}  // extern "C"
