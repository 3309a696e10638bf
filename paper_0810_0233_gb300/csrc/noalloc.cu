// noalloc.cu -- an entry point that allocates no memory: the FP64 direct
// field together with the energy E = -1/2 sum_i m_i . H_i, for callers that
// cannot call cudaMalloc (for example code that runs inside a host
// application whose GPU memory is owned by someone else's pool, or a plugin
// that must not change the device's allocation state).
//
// The per-block partial sums of m . H, which the other entry points keep in
// memory they allocate, live here in a file-scope __device__ array of fixed
// size.  Host code cannot use the array's name as a device address, so the
// address is fetched once per device with cudaGetSymbolAddress.
#include "../../include/ccfmm.h"
#include "ccfmm_dev.cuh"

#include <mutex>
#include <string>

namespace ccfmm {

constexpr int NA_T = 128;                       // threads per block
constexpr long long NA_MAX_BLOCKS = 32768;      // partial-sum slots
constexpr long long NA_MAX_N = NA_MAX_BLOCKS * NA_T;  // 4,194,304 dipoles

// slots [0, NA_MAX_BLOCKS): per-block partial sums; slot NA_MAX_BLOCKS: E
static __device__ __align__(256) double g_na_scratch[NA_MAX_BLOCKS + 1];

constexpr int NA_MAX_DEVICES = 64;
static double *g_na_ptr[NA_MAX_DEVICES];
static std::mutex g_na_mutex;

// Direct field at every dipole (j == i and r == 0 skipped, FP64), and the
// block's sum of m_i . H_i written to partial[blockIdx.x].
__global__ void __launch_bounds__(NA_T) k_direct_energy(const double *pos, const double *mom,
                                                        long long n, double *Hout,
                                                        double *partial)
{
    __shared__ double sp[256][6];
    __shared__ double red[NA_T / 32];
    long long i = (long long)blockIdx.x * NA_T + threadIdx.x;
    double xi = 0, yi = 0, zi = 0;
    if (i < n) {
        xi = pos[3 * i];
        yi = pos[3 * i + 1];
        zi = pos[3 * i + 2];
    }
    double hx = 0, hy = 0, hz = 0;
    for (long long b = 0; b < n; b += 256) {
        __syncthreads();
        for (int j = threadIdx.x; j < 256; j += NA_T) {
            long long q = b + j;
            if (q < n)
                for (int c = 0; c < 3; ++c) {
                    sp[j][c] = pos[3 * q + c];
                    sp[j][3 + c] = mom[3 * q + c];
                }
        }
        __syncthreads();
        int m = (int)min((long long)256, n - b);
        for (int j = 0; j < m; ++j) {
            if (b + j == i) continue;
            double rx = xi - sp[j][0], ry = yi - sp[j][1], rz = zi - sp[j][2];
            double r2 = rx * rx + ry * ry + rz * rz;
            if (r2 == 0.0) continue;
            double ri = 1.0 / sqrt(r2);
            double ri3 = ri * ri * ri;
            double mr = sp[j][3] * rx + sp[j][4] * ry + sp[j][5] * rz;
            double t3 = 3.0 * mr * ri * ri * ri3;
            hx += t3 * rx - sp[j][3] * ri3;
            hy += t3 * ry - sp[j][4] * ri3;
            hz += t3 * rz - sp[j][5] * ri3;
        }
    }
    double e = 0.0;
    if (i < n) {
        Hout[3 * i] = hx;
        Hout[3 * i + 1] = hy;
        Hout[3 * i + 2] = hz;
        e = mom[3 * i] * hx + mom[3 * i + 1] * hy + mom[3 * i + 2] * hz;
    }
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NA_T / 32; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// E = -1/2 * sum of partial[0 .. nparts), in a fixed order, into *E
__global__ void k_direct_energy_final(const double *partial, long long nparts, double *E)
{
    __shared__ double red[256];
    double t = 0.0;
    for (long long b = threadIdx.x; b < nparts; b += 256) t += partial[b];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = -0.5 * red[0];
}

}  // namespace ccfmm

using namespace ccfmm;

// Where a pointer lives, as this entry point needs it: memory that kernels
// on device dev can use directly (device memory of dev, or managed memory),
// memory of another device (never used: without peer access a kernel that
// touched it could fault), or host memory (any other pointer).
enum NaWhere { NA_HOST = 0, NA_THIS_DEVICE = 1, NA_OTHER_DEVICE = 2 };

static NaWhere na_where(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return NA_HOST;
    }
    if (a.type == cudaMemoryTypeManaged) return NA_THIS_DEVICE;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? NA_THIS_DEVICE : NA_OTHER_DEVICE;
    return NA_HOST;
}

extern "C" {

ccfmm_status ccfmm_direct_field_energy_noalloc(const double *positions, const double *moments,
                                               int64_t N, double *H_out, double *E_out,
                                               void *stream)
{
    set_last_error("");
    if (!positions || !moments || !H_out || !E_out) {
        set_last_error("NULL argument");
        return CCFMM_ERR_ARG;
    }
    if (N < 1 || N > NA_MAX_N) {
        set_last_error("N out of range: this entry point accepts 1 <= N <= 4194304 (its "
                       "fixed scratch holds 32768 block sums)");
        return CCFMM_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        set_last_error("no usable current CUDA device");
        return CCFMM_ERR_CUDA;
    }
    // the call synchronises its stream, which a capturing stream forbids
    if (stream) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
            cudaGetLastError();
            set_last_error("stream query failed");
            return CCFMM_ERR_CUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) {
            set_last_error("the stream is being captured: this call synchronises its stream");
            return CCFMM_ERR_ARG;
        }
    }
    if (na_where(positions, dev) != NA_THIS_DEVICE || na_where(moments, dev) != NA_THIS_DEVICE ||
        na_where(H_out, dev) != NA_THIS_DEVICE) {
        set_last_error((std::string("positions, moments and H_out must be device memory of the "
                                    "current device (device ") +
                        std::to_string(dev) + ")").c_str());
        return CCFMM_ERR_ARG;
    }
    const NaWhere e_where = na_where(E_out, dev);
    if (e_where == NA_OTHER_DEVICE) {
        set_last_error((std::string("E_out must be host memory or device memory of the current "
                                    "device (device ") +
                        std::to_string(dev) + ")").c_str());
        return CCFMM_ERR_ARG;
    }
    double *scratch = nullptr;
    {
        // set-up, once per device, with that device current: the device
        // address of the scratch array
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_ptr[dev]) {
            e = cudaGetSymbolAddress((void **)&g_na_ptr[dev], g_na_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                g_na_ptr[dev] = nullptr;
                set_last_error((std::string("cudaGetSymbolAddress failed: ") +
                                cudaGetErrorString(e)).c_str());
                return CCFMM_ERR_CUDA;
            }
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    long long nb = (N + NA_T - 1) / NA_T;
    // every slot the final reduction reads is written by this call's first
    // kernel, so nothing left from an earlier call is read
    note_launch(2);
    k_direct_energy<<<(unsigned)nb, NA_T, 0, s>>>(positions, moments, N, H_out, scratch);
    k_direct_energy_final<<<1, 256, 0, s>>>(scratch, nb, scratch + NA_MAX_BLOCKS);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E_out, scratch + NA_MAX_BLOCKS, sizeof(double),
                            e_where == NA_THIS_DEVICE ? cudaMemcpyDeviceToDevice
                                                      : cudaMemcpyDeviceToHost,
                            s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error((std::string("CUDA error: ") + cudaGetErrorString(e)).c_str());
        return CCFMM_ERR_CUDA;
    }
    return CCFMM_OK;
}

}  // extern "C"
