// Output-row reductions without any device allocation.
//
// dae_reduce_rows_noalloc computes the same sums as the row-reduction step of
// dae_assemble_reduced (J^T a_dense, J^T M J, J^T M dJ over the N output rows)
// from J, dJ and H[Delta,Delta] that the caller already holds on the device.
// Its per-block partial sums live in a fixed file-scope __device__ array instead
// of memory from cudaMalloc, for callers that cannot allocate: code running
// under a memory budget that forbids new device allocations after start-up,
// allocators that must not be re-entered, or hosts that own all device memory
// themselves.
//
// The array below is reserved on every GPU that loads this library, for the
// life of the process.  Its size bounds the problem: ceil(N / 128) blocks x
// (r + r(r+1)/2 + r^2) partials must fit in kNoAllocFloats.
#include <mutex>
#include <stdio.h>

#include "dae_internal.h"

namespace dae {

constexpr size_t kNoAllocFloats = (size_t)1 << 20;   // 4 MiB of FP32 partials
constexpr size_t kNoAllocDoubles = 4096;             // FP64 column sums
constexpr int kNoAllocMaxDevices = 64;
constexpr int NA_ROWS = 128;

static __device__ __align__(256) float g_noalloc_part[kNoAllocFloats];
static __device__ __align__(256) double g_noalloc_sum[kNoAllocDoubles];

// Per-block partials: [J^T a (r) | J^T M J upper (r(r+1)/2) | J^T M dJ (r*r, i*r+j)],
// a_n = m_n (sum_j J_nj z_j + H[D,D]_n) - dt^2 f_ext,n.
__global__ void __launch_bounds__(256) k_rows_noalloc(const float* J, const float* dJ,
                                                      const float* HDD, const float* mdof,
                                                      const float* f_ext, const float* z, int N,
                                                      int r, double dt, float* part, int stride) {
    __shared__ float Js[kMaxR][NA_ROWS + 1];
    __shared__ float dJs[kMaxR][NA_ROWS + 1];
    __shared__ float ms[NA_ROWS], as[NA_ROWS];
    const int t = threadIdx.x;
    const int n0 = blockIdx.x * NA_ROWS;
    if (t < NA_ROWS) {
        const int n = n0 + t;
        float m = 0.f, a = 0.f;
        if (n < N) {
            m = mdof[n];
            float y = HDD[n];
            for (int j = 0; j < r; ++j) {
                const float Jv = J[(size_t)j * N + n];
                Js[j][t] = Jv;
                dJs[j][t] = dJ[(size_t)j * N + n];
                y = fmaf(Jv, z[j], y);
            }
            a = (float)((double)m * y - dt * dt * (f_ext ? (double)f_ext[n] : 0.0));
        } else {
            for (int j = 0; j < r; ++j) { Js[j][t] = 0.f; dJs[j][t] = 0.f; }
        }
        ms[t] = m;
        as[t] = a;
    }
    __syncthreads();
    const int nsym = r * (r + 1) / 2;
    const int n_ent = r + nsym + r * r;
    float* out = part + (size_t)blockIdx.x * stride;
    for (int e = t; e < n_ent; e += blockDim.x) {
        float acc = 0.f;
        if (e < r) {
            for (int k = 0; k < NA_ROWS; ++k) acc = fmaf(Js[e][k], as[k], acc);
        } else if (e < r + nsym) {
            int p = e - r, i = 0;
            while (p >= r - i) { p -= r - i; ++i; }
            const int j = i + p;
            for (int k = 0; k < NA_ROWS; ++k) acc = fmaf(ms[k] * Js[i][k], Js[j][k], acc);
        } else {
            const int p = e - r - nsym, i = p / r, j = p % r;
            for (int k = 0; k < NA_ROWS; ++k) acc = fmaf(ms[k] * Js[i][k], dJs[j][k], acc);
        }
        out[e] = acc;
    }
}

// sum[e] = sum over blocks of part[b][e] in FP64 (32 threads per entry, fixed tree)
__global__ void k_rows_noalloc_sum(const float* part, int n_parts, int stride, int n_ent,
                                   double* sum) {
    const int e = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= n_ent) return;
    double acc = 0.0;
    for (int p = lane; p < n_parts; p += 32) acc += (double)part[(size_t)p * stride + e];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) sum[e] = acc;
}

// unpack into the caller's outputs (r x r matrices column-major)
__global__ void k_rows_noalloc_unpack(const double* sum, int r, double* phi, double* Mr, double* B) {
    const int nsym = r * (r + 1) / 2;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int i = e % r, j = e / r;
        const int a = i < j ? i : j, b = i < j ? j : i;
        if (Mr) Mr[e] = sum[r + a * r - a * (a - 1) / 2 + (b - a)];
        if (B) B[e] = sum[r + nsym + i * r + j];
    }
    if (phi)
        for (int i = threadIdx.x; i < r; i += blockDim.x) phi[i] = sum[i];
}

namespace {
std::mutex g_na_mu;
float* g_na_part_ptr[kNoAllocMaxDevices] = {};
double* g_na_sum_ptr[kNoAllocMaxDevices] = {};
}  // namespace

}  // namespace dae

using namespace dae;

extern "C" dae_status dae_reduce_rows_noalloc(int N, int r, const float* J, const float* dJ,
                                              const float* HDD, const float* mdof,
                                              const float* f_ext, const float* z, double dt,
                                              double* phi_dense, double* Mr, double* B,
                                              void* cuda_stream) {
    if (N <= 0 || r <= 0 || r > kMaxR || !J || !dJ || !HDD || !mdof || !z || !(dt > 0))
        return DAE_ERR_INVALID_ARG;
    const int n_blocks = (N + NA_ROWS - 1) / NA_ROWS;
    const int nsym = r * (r + 1) / 2;
    const int stride = r + nsym + r * r;
    if ((size_t)n_blocks * stride > kNoAllocFloats || (size_t)stride > kNoAllocDoubles)
        return DAE_ERR_INVALID_ARG;   // beyond the fixed scratch: N / r too large
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        return DAE_ERR_CUDA;
    }
    float* part;
    double* sum;
    {
        // once per device, with that device current: device addresses of the arrays
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_part_ptr[dev]) {
            float* p = nullptr;
            double* s = nullptr;
            if (cudaGetSymbolAddress((void**)&p, g_noalloc_part) != cudaSuccess ||
                cudaGetSymbolAddress((void**)&s, g_noalloc_sum) != cudaSuccess) {
                cudaGetLastError();
                return DAE_ERR_CUDA;
            }
            g_na_part_ptr[dev] = p;
            g_na_sum_ptr[dev] = s;
        }
        part = g_na_part_ptr[dev];
        sum = g_na_sum_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_rows_noalloc<<<n_blocks, 256, 0, s>>>(J, dJ, HDD, mdof, f_ext, z, N, r, dt, part, stride);
    k_rows_noalloc_sum<<<(stride + 7) / 8, 256, 0, s>>>(part, n_blocks, stride, stride, sum);
    k_rows_noalloc_unpack<<<1, 256, 0, s>>>(sum, r, phi_dense, Mr, B);
    return cudaGetLastError() == cudaSuccess ? DAE_OK : DAE_ERR_CUDA;
}
