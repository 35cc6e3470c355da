// Operator apply that allocates no device memory (coil_apply_operator_static).
//
// The dense far operator is stored with a row pitch ld >= N, and the apply
// kernels read an input vector that is ld long and zero beyond N.  The
// regular path keeps that padded copy in per-handle buffers; this entry keeps
// it in one file-scope device array instead, so a call needs no allocation at
// all: the caller passes its own N-long device input and output.
//
// The array is kStaticMaxLd = 2^20 doubles (8 MiB) in every device that loads
// the library, held until the process exits.  All calls share it and it keeps
// the last call's contents; the padding past N is cleared on every call.
// Two calls that overlap on the GPU (different streams, or different handles
// on the same device at the same time) race on it.
#include <mutex>

#include "../../include/coil.h"
#include "common.cuh"
#include "internal.h"

namespace cq {

constexpr long long kStaticMaxLd = 1LL << 20;

static __device__ __align__(256) double g_apply_scratch[kStaticMaxLd];

namespace {

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of the scratch array on `device` (which must be current).
// In host code the array's name is only a host-side stand-in, so the real
// address is looked up once per device and cached.
cudaError_t scratch_address(int device, double** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

}  // namespace

// Padded operator input: out[i] = p[i] for i < N, 0 for N <= i < ld.
template <typename T>
__global__ void k_static_pad(const double* __restrict__ p, int N, long long ld, T* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ld;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = i < N ? (T)p[i] : (T)0;
}

__device__ __forceinline__ float static_bf16(unsigned short v) { return __uint_as_float((unsigned)v << 16); }

// Entries a lane adds into its inner FP32 partial before folding it into the
// outer one (two FP32 levels, as the regular FP32/BF16 apply keeps them, so
// that the rounding does not grow with the row length).
constexpr int kStaticFold = 16;

// y = M_far p (one warp per row; FP64 storage multiplies in FP64, FP32/BF16
// storage in FP32 with two levels of FP32 lane partials and an FP64 warp
// reduction).
__global__ void k_static_far(const CoilDev* __restrict__ cds, const void* __restrict__ pin,
                             double* __restrict__ y) {
    const CoilDev& c = cds[0];
    int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (row >= c.N) return;
    double s = 0.0;
    if (c.precision == PREC_FP64) {
        const double* M = static_cast<const double*>(c.Mfar) + (size_t)row * c.ld;
        const double* p = static_cast<const double*>(pin);
        for (long long j = lane; j < c.ld; j += 32) s = fma(M[j], p[j], s);
    } else {
        const float* p = static_cast<const float*>(pin);
        const bool f32 = c.precision == PREC_FP32;
        const float* M32 = static_cast<const float*>(c.Mfar) + (size_t)row * c.ld;
        const unsigned short* M16 = static_cast<const unsigned short*>(c.Mfar) + (size_t)row * c.ld;
        float f = 0.f, outer = 0.f;
        int k = 0;
        for (long long j = lane; j < c.ld; j += 32) {
            float m = f32 ? M32[j] : static_bf16(M16[j]);
            f = fmaf(m, p[j], f);
            if (++k == kStaticFold) {
                outer += f;
                f = 0.f;
                k = 0;
            }
        }
        s = (double)outer + (double)f;
    }
    s = warp_sum(s);
    if (lane == 0) y[row] = s;
}

// y_w += M_ww p_w with the FP64 intra-wire blocks (one warp per block).
__global__ void k_static_near(const CoilDev* __restrict__ cds, const double* __restrict__ p,
                              double* __restrict__ y) {
    const CoilDev& c = cds[0];
    int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (w >= c.W) return;
    int B = c.B;
    const double* nb = c.near + (size_t)c.block_type[w] * B * B;
    const double* pw = p + (size_t)w * B;
    for (int i = lane; i < B; i += 32) {
        double acc = 0.0;
        for (int j = 0; j < B; ++j) acc += nb[i * B + j] * pw[j];
        y[w * B + i] += acc;
    }
}

}  // namespace cq

extern "C" coil_status coil_apply_operator_static(coil_t* c, const double* d_p, double* d_y, void* stream) {
    using namespace cq;
    CoilView v;
    if (!coil_view(c, &v)) return COIL_ERR_INVALID;
    if (!d_p || !d_y) return coil_set_error(c, COIL_ERR_INVALID, "apply_operator_static: null device buffer");
    const CoilDev& h = *v.host;
    if (h.op_format != 0)
        return coil_set_error(c, COIL_ERR_INVALID, "apply_operator_static: dense operator format only");
    if (h.ld > kStaticMaxLd)
        return coil_set_error(c, COIL_ERR_INVALID,
                              "apply_operator_static: operator pitch exceeds the static scratch "
                              "(at most 1048576 elements)");
    cudaError_t e = cudaSetDevice(v.device);
    double* scratch = nullptr;
    if (e == cudaSuccess) e = scratch_address(v.device, &scratch);
    if (e != cudaSuccess) return coil_set_error(c, COIL_ERR_CUDA, "apply_operator_static: set-up failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long ld = h.ld;
    unsigned pb = (unsigned)((ld + 255) / 256);
    if (pb > 4096u) pb = 4096u;
    if (h.precision == PREC_FP64)
        k_static_pad<double><<<pb, 256, 0, s>>>(d_p, h.N, ld, scratch);
    else
        k_static_pad<float><<<pb, 256, 0, s>>>(d_p, h.N, ld, reinterpret_cast<float*>(scratch));
    k_static_far<<<(unsigned)((h.N + 7) / 8), 256, 0, s>>>(v.dev, scratch, d_y);
    k_static_near<<<(unsigned)((h.W + 7) / 8), 256, 0, s>>>(v.dev, d_p, d_y);
    e = cudaGetLastError();
    if (e != cudaSuccess) return coil_set_error(c, COIL_ERR_CUDA, "apply_operator_static: launch failed");
    return COIL_OK;
}
