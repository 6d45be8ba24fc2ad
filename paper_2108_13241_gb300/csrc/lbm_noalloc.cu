// lbm_noalloc.cu -- lbm_reduce_f_noalloc: mass and momentum of a canonical
// distribution array with no memory allocation at all.
//
// Who needs it: callers that cannot call cudaMalloc (or any allocator) at the
// moment they want the reduction -- code running while a CUDA stream is being
// captured into a graph, a plugin whose host application owns every device
// buffer and hands out only fixed input/output buffers, or a real-time loop
// that must never enter the allocator.  The regular lbm_reduce takes its
// scratch from the workspace of an lbm_ctx; this entry point needs no
// context and no workspace: its scratch is the file-scope array below, which
// every GPU that loads the library keeps until the process exits.
//
// Scratch: one partial sum (4 doubles) per node row plus 4 doubles of result
// staging, for at most LBM_NOALLOC_MAX_ROWS rows: 16384 * 32 B + 256 B
// = 512.25 KiB per device.  Every partial is overwritten by each call before
// it is read, so nothing needs clearing between calls; calls that overlap on
// the GPU (two streams, or two host threads) share the array and race.
#include <cmath>
#include <mutex>

#include "lbm_internal.h"

namespace {

constexpr int NA_BLOCK = 256;
constexpr int NA_MAX_DEVICES = 64;

// partial[row][4] followed by 4 doubles of staging for the final sum
static __device__ __align__(256) double lbm_noalloc_scratch[LBM_NOALLOC_MAX_ROWS * 4 + 32];

std::mutex g_setup_mutex;
double *g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol's host-side shadow as a device
// pointer).  The cached address belongs to the device's context at the time
// of the first call; it does not survive cudaDeviceReset.
cudaError_t scratch_on_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, lbm_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__device__ __forceinline__ void na_block_sum4(double v[4], double *out) {
    __shared__ double sm[4][NA_BLOCK / 32];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) sm[c][w] = v[c];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < NA_BLOCK / 32; ++k) s += sm[c][k];
            out[c] = s;
        }
}

// One block per node row: sum over the row's included nodes of
// (sum_i f_i, sum_i c_ix f_i, sum_i c_iy f_i) in FP64.
template <class C>
__global__ void __launch_bounds__(NA_BLOCK) k_row_sums(const C *f, const uint8_t *mask, int nx, long long nnode,
                                                      double *partial) {
    const int y = blockIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int x = threadIdx.x; x < nx; x += NA_BLOCK) {
        const long long n = (long long)y * nx + x;
        if (mask && mask[n] == 0xFF) continue;
        double v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = (double)f[i * nnode + n];
        acc[0] += (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
        acc[1] += ((v[1] - v[3]) + (v[5] - v[7])) + (v[8] - v[6]);
        acc[2] += ((v[2] - v[4]) + (v[5] - v[7])) + (v[6] - v[8]);
    }
    na_block_sum4(acc, partial + 4 * (long long)y);
}

// Fixed-order sum of the row partials into out[0..2].
__global__ void __launch_bounds__(NA_BLOCK) k_rows_total(const double *partial, int rows, double *staging,
                                                        double *out) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r = threadIdx.x; r < rows; r += NA_BLOCK)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += partial[4 * r + c];
    na_block_sum4(acc, staging);
    if (threadIdx.x == 0) {
        out[0] = staging[0];
        out[1] = staging[1];
        out[2] = staging[2];
    }
}

} // namespace

extern "C" lbm_status lbm_reduce_f_noalloc(lbm_precision precision, const void *d_f, const uint8_t *d_mask,
                                           int nx, int ny, double *d_out, void *stream) {
    if (!d_f || !d_out || nx < 1 || ny < 1) return LBM_ERR_INVALID;
    if (ny > LBM_NOALLOC_MAX_ROWS) return LBM_ERR_INVALID; // beyond the static scratch
    if (precision != LBM_F64 && precision != LBM_F32 && precision != LBM_F16S) return LBM_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the scratch address is the current device's: the stream must belong to
    // that device too, or the kernels would write another GPU's scratch
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    if (sdev != dev) return LBM_ERR_INVALID;
    double *scratch = nullptr;
    if (scratch_on_current_device(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    // an error left behind by an earlier, unrelated call is not this call's
    cudaGetLastError();
    const long long nnode = (long long)nx * ny;
    double *partial = scratch;
    double *staging = scratch + (long long)LBM_NOALLOC_MAX_ROWS * 4;
    if (precision == LBM_F64)
        k_row_sums<double><<<ny, NA_BLOCK, 0, s>>>(static_cast<const double *>(d_f), d_mask, nx, nnode, partial);
    else
        k_row_sums<float><<<ny, NA_BLOCK, 0, s>>>(static_cast<const float *>(d_f), d_mask, nx, nnode, partial);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    k_rows_total<<<1, NA_BLOCK, 0, s>>>(partial, ny, staging, d_out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
