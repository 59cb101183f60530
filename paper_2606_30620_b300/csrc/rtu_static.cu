// rtu_static.cu -- rtu_gp_source_static: the GP source step (Eq. 1-3) without a
// caller-provided workspace, for callers that cannot allocate device memory.
//
// Its scratch is one file-scope __device__ array (RTU_STATIC_MAX_NSRC^2 complex
// floats, 128 KiB) that every GPU loading this library holds until the process
// exits.  Host code cannot pass the array's name to a kernel: in host code that
// name is a host-side stand-in, not a device address.  The first call on a
// device therefore looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and keeps it for later calls.
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
static __device__ __align__(256) float2 g_gp_static_scratch[SMAX * SMAX];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

rtu_status fail_static(rtu_status code, const std::string& m) { return rtu_fail_internal(code, m.c_str()); }

// One CTA: twiddles, digit reversal and radices built in shared memory, then
// the forward FFT, the sqrt(P) filter, the inverse FFT and the softplus map --
// the same device functions as the workspace path.
__global__ void __launch_bounds__(GP_NT) k_gp_source_static(int n, double pitch, int family, const float* lat,
                                                            const double* ps, float* out, Cx<float>* W) {
    extern __shared__ __align__(128) unsigned char smem_static[];
    Cx<float>* sm = reinterpret_cast<Cx<float>*>(smem_static);
    __shared__ Cx<float> tw_s[SMAX];
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
        tw_s[i] = Cx<float>{(float)cos(ang), (float)sin(ang)};
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
    const int chunk = max(1, min(n, (int)(GP_SMEM / sizeof(Cx<float>)) / n));
    for (int i = threadIdx.x; i < n2; i += blockDim.x) W[i] = Cx<float>{lat[i], 0.0f};
    __syncthreads();
    fft2<float>(W, n, rad_s, S, tw_s, rev_s, sm, chunk, false);
    const int nf = n_family(family);
    float psv[4];
    for (int q = 0; q < nf; ++q) psv[q] = (float)ps[q];
    const float kscale = (float)(2.0 * 3.14159265358979323846 / pitch);
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int ky = i / n, kx = i - ky * n;
        const float fx = fftfreq<float>(kx, n), fy = fftfreq<float>(ky, n);
        const float k = kscale * sqrtf(fx * fx + fy * fy);
        float gdummy[3];
        const float sp = sqrtP_and_grad<float>(family, psv, k, gdummy);
        W[i] = Cx<float>{W[i].x * sp, W[i].y * sp};
    }
    __syncthreads();
    fft2<float>(W, n, rad_s, S, tw_s, rev_s, sm, chunk, true);
    const float alpha = (float)ps[nf];
    const float inv_n2 = 1.0f / (float)n2;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const float f = W[i].x * inv_n2;
        out[i] = r_exp(alpha * log_sp_s0<float>(f / 0.01f));
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
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_scratch_addr[dev]) {
            // first call on this device (the device is current): device address of the
            // static array and the kernel's shared-memory limit
            void* p = nullptr;
            ce = cudaGetSymbolAddress(&p, g_gp_static_scratch);
            if (ce != cudaSuccess)
                return fail_static(RTU_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
            ce = cudaFuncSetAttribute(k_gp_source_static, cudaFuncAttributeMaxDynamicSharedMemorySize, GP_SMEM);
            if (ce != cudaSuccess)
                return fail_static(RTU_E_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce));
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    k_gp_source_static<<<1, GP_NT, GP_SMEM, static_cast<cudaStream_t>(stream)>>>(
        n_src, src_pitch, ps_family, latents, ps, source, static_cast<Cx<float>*>(scratch));
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail_static(RTU_E_CUDA, std::string("launch: ") + cudaGetErrorString(ce));
    return RTU_OK;
}

}  // extern "C"
