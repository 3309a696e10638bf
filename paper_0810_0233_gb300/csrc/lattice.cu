// lattice.cu -- the dipolar field of a simple-cubic lattice by FFT
// convolution, the comparator of Sec. V (the paper times the Cartesian FMM
// against an FFT method on its lattice benchmark of Sec. IV).
//
// On a lattice r_i = a (ix, iy, iz) the field of Eq. H2 (as read),
//     H_i = sum_{j != i} G(r_i - r_j) m_j,
//     G(r) = (3 r r^T - |r|^2 I) / |r|^5,  G(0) = 0,
// is a discrete 3-D convolution of the moments with the 3 x 3 symmetric
// tensor G sampled at integer offsets.  With every axis zero-padded to
// P = 2n (n = 1: P = 1) the cyclic convolution of the padded grids equals the
// open-boundary sum (offsets reach -(n-1) .. n-1, and no wrapped copy
// overlaps).  Per evaluation:
//   scatter   moments into three padded real grids (zeros elsewhere),
//   forward   three real-to-complex 3-D FFTs (cuFFT),
//   multiply  H^_a = sum_b G^_ab M^_b per frequency (six tensor spectra,
//             transformed once per handle),
//   inverse   three complex-to-real FFTs,
//   gather    H at the lattice points, divided by P1 P2 P3, and the energy
//             E = -1/2 sum m.H (fixed-order FP64 reduction).
// The FFTs are library calls; cuFFT is opened at run time (dlopen) by the
// first handle, so the rest of the library does not depend on it.
#include "../../include/ccfmm.h"
#include "ccfmm_dev.cuh"

#include <cufft.h>
#include <dlfcn.h>

#include <cmath>
#include <mutex>
#include <string>

namespace ccfmm {

// ---------------------------------------------------------------- cuFFT
struct CufftApi {
    bool ok = false;
    std::string why;
    cufftResult (*plan_many)(cufftHandle *, int, int *, int *, int, int, int *, int, int,
                             cufftType, int) = nullptr;
    cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
    cufftResult (*destroy)(cufftHandle) = nullptr;
    cufftResult (*exec_r2c)(cufftHandle, cufftReal *, cufftComplex *) = nullptr;
    cufftResult (*exec_c2r)(cufftHandle, cufftComplex *, cufftReal *) = nullptr;
    cufftResult (*exec_d2z)(cufftHandle, cufftDoubleReal *, cufftDoubleComplex *) = nullptr;
    cufftResult (*exec_z2d)(cufftHandle, cufftDoubleComplex *, cufftDoubleReal *) = nullptr;
};

static const CufftApi &cufft_api()
{
    static CufftApi api;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libcufft.so.12", "libcufft.so", "/usr/local/cuda/lib64/libcufft.so.12",
                               "/usr/local/cuda/lib64/libcufft.so"};
        void *lib = nullptr;
        for (const char *n : names)
            if ((lib = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
        if (!lib) {
            api.why = "cuFFT (libcufft.so) could not be opened";
            return;
        }
        auto sym = [&](const char *n) { return dlsym(lib, n); };
        api.plan_many = reinterpret_cast<decltype(api.plan_many)>(sym("cufftPlanMany"));
        api.set_stream = reinterpret_cast<decltype(api.set_stream)>(sym("cufftSetStream"));
        api.destroy = reinterpret_cast<decltype(api.destroy)>(sym("cufftDestroy"));
        api.exec_r2c = reinterpret_cast<decltype(api.exec_r2c)>(sym("cufftExecR2C"));
        api.exec_c2r = reinterpret_cast<decltype(api.exec_c2r)>(sym("cufftExecC2R"));
        api.exec_d2z = reinterpret_cast<decltype(api.exec_d2z)>(sym("cufftExecD2Z"));
        api.exec_z2d = reinterpret_cast<decltype(api.exec_z2d)>(sym("cufftExecZ2D"));
        api.ok = api.plan_many && api.set_stream && api.destroy && api.exec_r2c && api.exec_c2r &&
                 api.exec_d2z && api.exec_z2d;
        if (!api.ok) api.why = "cuFFT lacks an expected entry point";
    });
    return api;
}

template <typename real> struct Cplx;
template <> struct Cplx<float> { typedef float2 t; };
template <> struct Cplx<double> { typedef double2 t; };

struct LatDims {
    int n[3];   // lattice points per axis
    int P[3];   // padded grid
    int Ph;     // P[2] / 2 + 1 (last axis of the spectra)
    double a;   // spacing
};

// grid offset along one axis: g < n -> g; g > P - n -> g - P; else outside
__device__ __forceinline__ bool lat_offset(int g, int n, int P, int &d)
{
    if (g < n) {
        d = g;
        return true;
    }
    if (g > P - n) {
        d = g - P;
        return true;
    }
    return false;
}

// six components xx, xy, xz, yy, yz, zz of G at every grid offset, FP64
// arithmetic, stored in the transform precision
template <typename real>
__global__ void k_lat_kernel(LatDims D, real *G)
{
    const long long np = (long long)D.P[0] * D.P[1] * D.P[2];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= np) return;
    const int gz = (int)(g % D.P[2]);
    const int gy = (int)((g / D.P[2]) % D.P[1]);
    const int gx = (int)(g / ((long long)D.P[2] * D.P[1]));
    int dx, dy, dz;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (lat_offset(gx, D.n[0], D.P[0], dx) && lat_offset(gy, D.n[1], D.P[1], dy) &&
        lat_offset(gz, D.n[2], D.P[2], dz) && (dx | dy | dz)) {
        const double x = D.a * dx, y = D.a * dy, z = D.a * dz;
        const double r2 = x * x + y * y + z * z;
        const double ri2 = 1.0 / r2;
        const double ri3 = ri2 / sqrt(r2);
        const double t = 3.0 * ri2;
        v[0] = ri3 * (t * x * x - 1.0);
        v[1] = ri3 * (t * x * y);
        v[2] = ri3 * (t * x * z);
        v[3] = ri3 * (t * y * y - 1.0);
        v[4] = ri3 * (t * y * z);
        v[5] = ri3 * (t * z * z - 1.0);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) G[c * np + g] = (real)v[c];
}

// padded moment grids (three components), zeros outside the lattice
template <typename real>
__global__ void k_lat_scatter(LatDims D, const double *mom, real *M)
{
    const long long np = (long long)D.P[0] * D.P[1] * D.P[2];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= np) return;
    const int gz = (int)(g % D.P[2]);
    const int gy = (int)((g / D.P[2]) % D.P[1]);
    const int gx = (int)(g / ((long long)D.P[2] * D.P[1]));
    real m[3] = {(real)0, (real)0, (real)0};
    if (gx < D.n[0] && gy < D.n[1] && gz < D.n[2]) {
        const long long i = ((long long)gx * D.n[1] + gy) * D.n[2] + gz;
        m[0] = (real)mom[3 * i];
        m[1] = (real)mom[3 * i + 1];
        m[2] = (real)mom[3 * i + 2];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) M[c * np + g] = m[c];
}

// H^_a = sum_b G^_ab M^_b per frequency, written over M^
template <typename real>
__global__ void k_lat_multiply(long long nf, const typename Cplx<real>::t *Gh,
                               typename Cplx<real>::t *Mh)
{
    typedef typename Cplx<real>::t C2;
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const C2 m0 = Mh[f], m1 = Mh[nf + f], m2 = Mh[2 * nf + f];
    C2 g[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) g[c] = Gh[c * nf + f];
    // symmetric tensor: rows (xx xy xz) (xy yy yz) (xz yz zz)
    const int row[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    const C2 mm[3] = {m0, m1, m2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        real re = 0, im = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const C2 gg = g[row[a][b]];
            re += gg.x * mm[b].x - gg.y * mm[b].y;
            im += gg.x * mm[b].y + gg.y * mm[b].x;
        }
        C2 o;
        o.x = re;
        o.y = im;
        Mh[a * nf + f] = o;
    }
}

constexpr int LAT_T = 256;

// H at the lattice points (input order), scaled by 1 / (P1 P2 P3), and
// per-block partial sums of m.H
template <typename real>
__global__ void __launch_bounds__(LAT_T) k_lat_gather(LatDims D, const real *Hg,
                                                      const double *mom, double *H_out,
                                                      double *partial)
{
    __shared__ double red[LAT_T / 32];
    const long long np = (long long)D.P[0] * D.P[1] * D.P[2];
    const long long n = (long long)D.n[0] * D.n[1] * D.n[2];
    const long long i = (long long)blockIdx.x * LAT_T + threadIdx.x;
    double e = 0.0;
    if (i < n) {
        const int iz = (int)(i % D.n[2]);
        const int iy = (int)((i / D.n[2]) % D.n[1]);
        const int ix = (int)(i / ((long long)D.n[2] * D.n[1]));
        const long long g = ((long long)ix * D.P[1] + iy) * D.P[2] + iz;
        const double sc = 1.0 / (double)np;
        const double h[3] = {sc * (double)Hg[g], sc * (double)Hg[np + g],
                             sc * (double)Hg[2 * np + g]};
        H_out[3 * i] = h[0];
        H_out[3 * i + 1] = h[1];
        H_out[3 * i + 2] = h[2];
        e = mom[3 * i] * h[0] + mom[3 * i + 1] * h[1] + mom[3 * i + 2] * h[2];
    }
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < LAT_T / 32; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_lat_energy(const double *partial, long long nparts, double *E)
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

struct ccfmm_lattice_s {
    LatDims D;
    int prec = CCFMM_FP64;
    cudaStream_t stream = nullptr;
    long long np = 0, nf = 0, n = 0;
    void *G = nullptr;      // six tensor spectra
    void *R = nullptr;      // three real grids (moments, then fields)
    void *Cx = nullptr;     // three spectra
    double *mom = nullptr;  // N x 3 copy of the moments
    double *H = nullptr;    // N x 3 field (host outputs are copied from it)
    double *part = nullptr; // energy partials, then E at the end
    int *flag = nullptr;    // device: non-finite moments seen
    int *hflag = nullptr;   // pinned host copy of the flag
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
};

static ccfmm_status lat_fail(ccfmm_status st, const std::string &msg)
{
    set_last_error(msg.c_str());
    return st;
}

#define LCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return lat_fail(CCFMM_ERR_CUDA, std::string(#call) + " failed: " +                   \
                                                cudaGetErrorString(e_));                         \
        }                                                                                        \
    } while (0)
#define LFF(call)                                                                                \
    do {                                                                                         \
        cufftResult r_ = (call);                                                                 \
        if (r_ != CUFFT_SUCCESS)                                                                 \
            return lat_fail(CCFMM_ERR_CUDA, std::string(#call) + " failed: cufftResult " +       \
                                                std::to_string((int)r_));                        \
    } while (0)

static bool lat_is_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void lat_free(ccfmm_lattice_t h)
{
    const CufftApi &api = cufft_api();
    if (h->have_fwd && api.ok) api.destroy(h->fwd);
    if (h->have_inv && api.ok) api.destroy(h->inv);
    cudaFree(h->G);
    cudaFree(h->R);
    cudaFree(h->Cx);
    cudaFree(h->mom);
    cudaFree(h->H);
    cudaFree(h->part);
    cudaFree(h->flag);
    cudaFreeHost(h->hflag);
    delete h;
}

template <typename real>
static ccfmm_status lat_plans(ccfmm_lattice_t h, const CufftApi &api)
{
    typedef typename Cplx<real>::t C2;
    const bool dp = sizeof(real) == 8;
    int dims[3] = {h->D.P[0], h->D.P[1], h->D.P[2]};
    const int idist = (int)h->np, odist = (int)h->nf;
    // tensor spectra: six forward transforms, once
    cufftHandle g6;
    LFF(api.plan_many(&g6, 3, dims, nullptr, 1, idist, nullptr, 1, odist,
                      dp ? CUFFT_D2Z : CUFFT_R2C, 6));
    cufftResult r = api.set_stream(g6, h->stream);
    const unsigned nb = (unsigned)((h->np + 255) / 256);
    note_launch();
    k_lat_kernel<real><<<nb, 256, 0, h->stream>>>(h->D, reinterpret_cast<real *>(h->R));
    // the six kernel grids live in R (sized for six) until their spectra exist
    if (r == CUFFT_SUCCESS)
        r = dp ? api.exec_d2z(g6, reinterpret_cast<cufftDoubleReal *>(h->R),
                              reinterpret_cast<cufftDoubleComplex *>(h->G))
               : api.exec_r2c(g6, reinterpret_cast<cufftReal *>(h->R),
                              reinterpret_cast<cufftComplex *>(h->G));
    cudaError_t e = cudaStreamSynchronize(h->stream);
    api.destroy(g6);
    LFF(r);
    LCK(e);
    LFF(api.plan_many(&h->fwd, 3, dims, nullptr, 1, idist, nullptr, 1, odist,
                      dp ? CUFFT_D2Z : CUFFT_R2C, 3));
    h->have_fwd = true;
    LFF(api.plan_many(&h->inv, 3, dims, nullptr, 1, odist, nullptr, 1, idist,
                      dp ? CUFFT_Z2D : CUFFT_C2R, 3));
    h->have_inv = true;
    LFF(api.set_stream(h->fwd, h->stream));
    LFF(api.set_stream(h->inv, h->stream));
    (void)sizeof(C2);
    return CCFMM_OK;
}

template <typename real>
static ccfmm_status lat_eval(ccfmm_lattice_t h, const CufftApi &api, double *Hdev, double *Edev)
{
    typedef typename Cplx<real>::t C2;
    const bool dp = sizeof(real) == 8;
    cudaStream_t s = h->stream;
    const unsigned nbp = (unsigned)((h->np + 255) / 256);
    note_launch();
    k_lat_scatter<real><<<nbp, 256, 0, s>>>(h->D, h->mom, reinterpret_cast<real *>(h->R));
    LCK(cudaGetLastError());
    if (dp)
        LFF(api.exec_d2z(h->fwd, reinterpret_cast<cufftDoubleReal *>(h->R),
                         reinterpret_cast<cufftDoubleComplex *>(h->Cx)));
    else
        LFF(api.exec_r2c(h->fwd, reinterpret_cast<cufftReal *>(h->R),
                         reinterpret_cast<cufftComplex *>(h->Cx)));
    note_launch();
    k_lat_multiply<real><<<(unsigned)((h->nf + 255) / 256), 256, 0, s>>>(
        h->nf, reinterpret_cast<const C2 *>(h->G), reinterpret_cast<C2 *>(h->Cx));
    LCK(cudaGetLastError());
    if (dp)
        LFF(api.exec_z2d(h->inv, reinterpret_cast<cufftDoubleComplex *>(h->Cx),
                         reinterpret_cast<cufftDoubleReal *>(h->R)));
    else
        LFF(api.exec_c2r(h->inv, reinterpret_cast<cufftComplex *>(h->Cx),
                         reinterpret_cast<cufftReal *>(h->R)));
    const long long nb = (h->n + LAT_T - 1) / LAT_T;
    note_launch(2);
    k_lat_gather<real><<<(unsigned)nb, LAT_T, 0, s>>>(h->D, reinterpret_cast<const real *>(h->R),
                                                      h->mom, Hdev, h->part);
    k_lat_energy<<<1, 256, 0, s>>>(h->part, nb, Edev);
    LCK(cudaGetLastError());
    return CCFMM_OK;
}

extern "C" {

ccfmm_status fmm_lattice_create(int32_t nx, int32_t ny, int32_t nz, double spacing,
                                int32_t precision, void *cuda_stream, ccfmm_lattice_t *out)
{
    set_last_error("");
    if (!out) return lat_fail(CCFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096)
        return lat_fail(CCFMM_ERR_ARG, "lattice sizes must lie in 1 .. 4096");
    if (!(spacing > 0.0) || !std::isfinite(spacing))
        return lat_fail(CCFMM_ERR_ARG, "spacing must be finite and > 0");
    if (precision != CCFMM_FP64 && precision != CCFMM_MIXED)
        return lat_fail(CCFMM_ERR_ARG, "precision must be CCFMM_FP64 or CCFMM_MIXED");
    const CufftApi &api = cufft_api();
    if (!api.ok) return lat_fail(CCFMM_ERR_CUDA, api.why);
    ccfmm_lattice_t h = new ccfmm_lattice_s;
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        h->D.n[a] = n[a];
        h->D.P[a] = n[a] == 1 ? 1 : 2 * n[a];
    }
    h->D.Ph = h->D.P[2] / 2 + 1;
    h->D.a = spacing;
    h->prec = precision;
    h->stream = (cudaStream_t)cuda_stream;
    h->n = (long long)nx * ny * nz;
    h->np = (long long)h->D.P[0] * h->D.P[1] * h->D.P[2];
    h->nf = (long long)h->D.P[0] * h->D.P[1] * h->D.Ph;
    if (6 * h->np >= (1ll << 31) || 6 * h->nf >= (1ll << 31)) {
        delete h;
        return lat_fail(CCFMM_ERR_ARG, "padded lattice too large for 32-bit FFT batch strides");
    }
    const size_t rs = precision == CCFMM_FP64 ? 8 : 4;
    const long long nb = (h->n + LAT_T - 1) / LAT_T;
    cudaError_t e = cudaMalloc(&h->G, 6 * 2 * rs * (size_t)h->nf);
    if (e == cudaSuccess) e = cudaMalloc(&h->R, 6 * rs * (size_t)h->np);
    if (e == cudaSuccess) e = cudaMalloc(&h->Cx, 3 * 2 * rs * (size_t)h->nf);
    if (e == cudaSuccess) e = cudaMalloc(&h->mom, 3 * sizeof(double) * (size_t)h->n);
    if (e == cudaSuccess) e = cudaMalloc(&h->H, 3 * sizeof(double) * (size_t)h->n);
    if (e == cudaSuccess) e = cudaMalloc(&h->part, sizeof(double) * (size_t)(nb + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&h->hflag, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        lat_free(h);
        return lat_fail(CCFMM_ERR_ALLOC, std::string("device allocation failed: ") +
                                             cudaGetErrorString(e));
    }
    ccfmm_status st = precision == CCFMM_FP64 ? lat_plans<double>(h, api) : lat_plans<float>(h, api);
    if (st != CCFMM_OK) {
        std::string msg = ccfmm_last_error();
        lat_free(h);
        return lat_fail(st, msg);
    }
    *out = h;
    return CCFMM_OK;
}

ccfmm_status fmm_lattice_field(ccfmm_lattice_t h, const double *moments, double *H_out,
                               double *E_out)
{
    set_last_error("");
    if (!h || !moments) return lat_fail(CCFMM_ERR_ARG, "NULL handle or moments");
    const CufftApi &api = cufft_api();
    cudaStream_t s = h->stream;
    const size_t bytes = 3 * sizeof(double) * (size_t)h->n;
    LCK(cudaMemcpyAsync(h->mom, moments, bytes,
                        lat_is_device(moments) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        s));
    LCK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    launch_check_finite(h->mom, 3 * h->n, h->flag, s);
    const bool h_dev = H_out && lat_is_device(H_out);
    double *Hdev = h_dev ? H_out : h->H;
    const long long nb = (h->n + LAT_T - 1) / LAT_T;
    double *Edev = h->part + nb;
    ccfmm_status st = h->prec == CCFMM_FP64 ? lat_eval<double>(h, api, Hdev, Edev)
                                            : lat_eval<float>(h, api, Hdev, Edev);
    if (st != CCFMM_OK) return st;
    if (H_out && !h_dev) LCK(cudaMemcpyAsync(H_out, Hdev, bytes, cudaMemcpyDeviceToHost, s));
    if (E_out)
        LCK(cudaMemcpyAsync(E_out, Edev, sizeof(double),
                            lat_is_device(E_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            s));
    LCK(cudaMemcpyAsync(h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    LCK(cudaStreamSynchronize(s));
    if (*h->hflag) return lat_fail(CCFMM_ERR_ARG, "moments contain non-finite values");
    return CCFMM_OK;
}

void fmm_lattice_destroy(ccfmm_lattice_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    lat_free(h);
}

}  // extern "C"
