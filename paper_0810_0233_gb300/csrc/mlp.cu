// mlp.cu -- the parameter selector (a project addition; the paper picks the
// leaf occupancy by Eq. so and (p_m, alpha_m) from Table II / Fig. 3 by
// hand): problem features of a dipole set, and a 12-64-64-64-2 MLP with BF16
// weights and FP32 accumulation that predicts (log10 time per dipole,
// log10 relative RMS error) of the FMM for (features, p, theta, leaf).
// Forward, backward and Adam are hand-written kernels.
#include "../../include/ccfmm.h"
#include "ccfmm_dev.cuh"

#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

namespace ccfmm {

constexpr int MIN_ = 12, MH = 64, MOUT = 2, NLAYER = 4;
constexpr int MLP_NP = MIN_ * MH + MH + 2 * (MH * MH + MH) + MH * MOUT + MOUT;  // 9282
constexpr int MLP_T = 128;

// parameter offsets: W1[12][64] b1 W2[64][64] b2 W3[64][64] b3 W4[64][2] b4
__host__ __device__ constexpr int off_w(int l)
{
    return l == 0 ? 0 : (l == 1 ? MIN_ * MH + MH : (l == 2 ? MIN_ * MH + MH + MH * MH + MH
                                                             : MIN_ * MH + MH + 2 * (MH * MH + MH)));
}
__host__ __device__ constexpr int dim_in(int l) { return l == 0 ? MIN_ : MH; }
__host__ __device__ constexpr int dim_out(int l) { return l == NLAYER - 1 ? MOUT : MH; }
__host__ __device__ constexpr int off_b(int l) { return off_w(l) + dim_in(l) * dim_out(l); }

// norm: mu_x[12] sd_x[12] mu_y[2] sd_y[2]
constexpr int NORM_N = 2 * MIN_ + 2 * MOUT;

__global__ void k_to_bf16(const float *w, __nv_bfloat16 *wb, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

// forward, one thread per row; activations live in shared memory rows of
// stride MH+1 (conflict-free); hidden activations (post-ReLU) are stored for
// the backward pass when H != nullptr; outputs in standardised units
constexpr int ACT_LD = MH + 1;

__global__ void __launch_bounds__(MLP_T) k_mlp_forward(const float *X, long long B,
                                                       const __nv_bfloat16 *wb, const float *norm,
                                                       float *Y, float *H)
{
    extern __shared__ float smf[];
    float *w = smf;                                  // [MLP_NP]
    float *act = smf + MLP_NP;                       // [2][MLP_T][ACT_LD]
    for (int i = threadIdx.x; i < MLP_NP; i += MLP_T) w[i] = __bfloat162float(wb[i]);
    __syncthreads();
    long long b = (long long)blockIdx.x * MLP_T + threadIdx.x;
    if (b >= B) return;
    float *a = act + threadIdx.x * ACT_LD;
    float *z = act + (MLP_T + threadIdx.x) * ACT_LD;
    for (int i = 0; i < MIN_; ++i) a[i] = (X[b * MIN_ + i] - norm[i]) / norm[MIN_ + i];
    for (int l = 0; l < NLAYER; ++l) {
        const int ni = dim_in(l), no = dim_out(l);
        const float *W = w + off_w(l), *bb = w + off_b(l);
        for (int o = 0; o < no; ++o) {
            float s = bb[o];
#pragma unroll 4
            for (int i = 0; i < ni; ++i) s += a[i] * W[i * no + o];
            if (l < NLAYER - 1) {
                s = fmaxf(s, 0.f);
                z[o] = s;
                if (H) H[((long long)l * B + b) * MH + o] = s;
            } else {
                Y[b * MOUT + o] = s;
            }
        }
        float *t = a;
        a = z;
        z = t;
    }
}

// dY = 2 mask (Y - T_n) / count, per-block loss partial sums
__global__ void k_mlp_loss(const float *Y, const float *T, const float *mask, long long B,
                           const float *norm, const float *count, float *dY, float *lpart)
{
    __shared__ float red[MLP_T];
    long long b = (long long)blockIdx.x * MLP_T + threadIdx.x;
    float l = 0.f;
    float c = fmaxf(*count, 1.f);
    if (b < B) {
        for (int o = 0; o < MOUT; ++o) {
            float tn = (T[b * MOUT + o] - norm[2 * MIN_ + o]) / norm[2 * MIN_ + MOUT + o];
            float m = mask[b * MOUT + o];
            float d = Y[b * MOUT + o] - tn;
            l += m * d * d;
            dY[b * MOUT + o] = 2.f * m * d / c;
        }
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int w = MLP_T / 2; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = red[0] / c;
}

// dZ_in[b][i] = (sum_o dZ[b][o] W[i][o]) * (A_in[b][i] > 0), one thread per row
__global__ void __launch_bounds__(MLP_T) k_mlp_back_rows(const float *dZ, int no,
                                                         const __nv_bfloat16 *W, const float *A,
                                                         long long B, float *dZin)
{
    __shared__ float w[MH * MH];
    __shared__ float dsh[MLP_T * ACT_LD];
    for (int i = threadIdx.x; i < MH * no; i += MLP_T) w[i] = __bfloat162float(W[i]);
    __syncthreads();
    long long b = (long long)blockIdx.x * MLP_T + threadIdx.x;
    if (b >= B) return;
    float *d = dsh + threadIdx.x * ACT_LD;
    for (int o = 0; o < no; ++o) d[o] = dZ[b * no + o];
    for (int i = 0; i < MH; ++i) {
        float s = 0.f;
#pragma unroll 4
        for (int o = 0; o < no; ++o) s += d[o] * w[i * no + o];
        dZin[b * MH + i] = A[b * MH + i] > 0.f ? s : 0.f;
    }
}

// gW[i][o] = sum_b A[b][i] dZ[b][o]; gb[o] = sum_b dZ[b][o].  Block (i-chunk,
// row-chunk); partial sums added with atomics.
constexpr int GW_ROWS = 2048;
__global__ void k_mlp_grad_w(const float *A, int ni, int lda, bool normalize_x, const float *norm,
                             const float *dZ, int no, long long B, float *gW, float *gb)
{
    long long r0 = (long long)blockIdx.y * GW_ROWS;
    long long r1 = min(B, r0 + GW_ROWS);
    int i = blockIdx.x;  // input index; i == ni computes the bias gradient
    for (int o = threadIdx.x; o < no; o += blockDim.x) {
        float s = 0.f;
        for (long long b = r0; b < r1; ++b) {
            float a = 1.f;
            if (i < ni) {
                a = A[b * lda + i];
                if (normalize_x) a = (a - norm[i]) / norm[MIN_ + i];
            }
            s += a * dZ[b * no + o];
        }
        if (i < ni)
            atomicAdd(&gW[i * no + o], s);
        else
            atomicAdd(&gb[o], s);
    }
}

__global__ void k_adam(float *w, const float *g, float *m1, float *m2, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float a = b1 * m1[i] + (1.f - b1) * gi;
    float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    w[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

// column mean / std of X (B x 12) and of the masked targets (B x 2)
__global__ void k_fit_norm(const float *X, const float *T, const float *mask, long long B,
                           float *norm)
{
    int c = threadIdx.x;  // 0..11 features, 12..13 targets
    if (c >= MIN_ + MOUT) return;
    double s = 0.0, s2 = 0.0, n = 0.0;
    for (long long b = 0; b < B; ++b) {
        double v, m = 1.0;
        if (c < MIN_) {
            v = X[b * MIN_ + c];
        } else {
            v = T[b * MOUT + c - MIN_];
            m = mask[b * MOUT + c - MIN_];
        }
        s += m * v;
        s2 += m * v * v;
        n += m;
    }
    double mu = n > 0 ? s / n : 0.0;
    double var = n > 0 ? s2 / n - mu * mu : 1.0;
    double sd = var > 1e-12 ? sqrt(var) : 1.0;
    if (c < MIN_) {
        norm[c] = (float)mu;
        norm[MIN_ + c] = (float)sd;
    } else {
        norm[2 * MIN_ + c - MIN_] = (float)mu;
        norm[2 * MIN_ + MOUT + c - MIN_] = (float)sd;
    }
}

__global__ void k_sum(const float *x, long long n, float *out)
{
    __shared__ float red[256];
    float s = 0.f;
    for (long long i = threadIdx.x; i < n; i += 256) s += x[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_destandardise(float *Y, long long B, const float *norm)
{
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B * MOUT) return;
    int o = (int)(j % MOUT);
    Y[j] = Y[j] * norm[2 * MIN_ + MOUT + o] + norm[2 * MIN_ + o];
}

// ---------------------------------------------------------------- features
// occupancy counts of the depth-Lr cells (keys are LCAP-bit bisection keys)
__global__ void k_cell_hist(const uint32_t *keys, long long n, int Lr, int *cnt)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[keys[i] >> (LCAP - Lr)], 1);
}

// raw moments of the counts: sum c, c^2, c^3, c^4 (FP64)
__global__ void k_count_moments(const int *cnt, long long ncell, double *mom4)
{
    __shared__ double red[4][256];
    double s[4] = {0, 0, 0, 0};
    for (long long k = (long long)blockIdx.x * 256 + threadIdx.x; k < ncell;
         k += (long long)gridDim.x * 256) {
        double c = cnt[k];
        s[0] += c;
        s[1] += c * c;
        s[2] += c * c * c;
        s[3] += c * c * c * c;
    }
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = 128; w; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) atomicAdd(&mom4[q], red[q][0]);
}

__global__ void k_to_f32(const double *pos, long long n, float4 *p4)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p4[i] = make_float4((float)pos[3 * i], (float)pos[3 * i + 1], (float)pos[3 * i + 2], 0.f);
}

// nearest-neighbour distance of S sample points (indices i*n/S) to all points
__global__ void __launch_bounds__(128) k_nn_sample(const float4 *p4, long long n, int S, float *nn)
{
    __shared__ float4 sp[512];
    int s = blockIdx.x * 128 + threadIdx.x;
    long long self = s < S ? (long long)s * n / S : -1;
    float4 me = s < S ? p4[self] : make_float4(0, 0, 0, 0);
    float best = INFINITY;
    for (long long b = 0; b < n; b += 512) {
        __syncthreads();
        for (int j = threadIdx.x; j < 512; j += 128)
            if (b + j < n) sp[j] = p4[b + j];
        __syncthreads();
        int m = (int)min((long long)512, n - b);
        for (int j = 0; j < m; ++j) {
            float dx = me.x - sp[j].x, dy = me.y - sp[j].y, dz = me.z - sp[j].z;
            float d2 = dx * dx + dy * dy + dz * dz;
            if (b + j != self) best = fminf(best, d2);
        }
    }
    if (s < S) nn[s] = sqrtf(best);
}

}  // namespace ccfmm

using namespace ccfmm;

static size_t fwd_smem()
{
    size_t b = sizeof(float) * ((size_t)MLP_NP + 2 * MLP_T * ACT_LD);
    static bool set = false;
    if (!set) {
        cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
        set = true;
    }
    return b;
}

struct ccfmm_mlp_s {
    int device = 0;
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr, *norm = nullptr;
    __nv_bfloat16 *wb = nullptr;
    float *work = nullptr;
    size_t work_bytes = 0;
    long long t = 0;
};

static ccfmm_status mlp_fail(ccfmm_status st, const std::string &m)
{
    set_last_error(m.c_str());
    return st;
}

#define MCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return mlp_fail(CCFMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
        }                                                                                        \
    } while (0)

static bool dev_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device copy of a host or device float array
struct FBuf {
    float *p = nullptr;
    bool own = false;
    ~FBuf()
    {
        if (own) cudaFree(p);
    }
};
static ccfmm_status fbuf(FBuf &b, const float *src, long long n)
{
    if (dev_ptr(src)) {
        b.p = const_cast<float *>(src);
        return CCFMM_OK;
    }
    MCK(cudaMalloc(&b.p, sizeof(float) * std::max(n, 1ll)));
    b.own = true;
    MCK(cudaMemcpy(b.p, src, sizeof(float) * n, cudaMemcpyHostToDevice));
    return CCFMM_OK;
}

static ccfmm_status mlp_work(ccfmm_mlp_t m, size_t bytes)
{
    if (m->work_bytes >= bytes) return CCFMM_OK;
    cudaFree(m->work);
    m->work = nullptr;
    m->work_bytes = 0;
    MCK(cudaMalloc(&m->work, bytes));
    m->work_bytes = bytes;
    return CCFMM_OK;
}

// forward + loss + backward; gradient left in m->g, loss returned
static ccfmm_status mlp_grad(ccfmm_mlp_t m, const float *X, const float *T, const float *mask,
                             long long B, float *loss)
{
    size_t need = sizeof(float) * ((size_t)B * (3 * MH + MOUT + MOUT + 2 * MH) + B / MLP_T + 8);
    ccfmm_status st = mlp_work(m, need);
    if (st != CCFMM_OK) return st;
    float *Hs = m->work;                   // [3][B][64]
    float *Y = Hs + 3 * (size_t)B * MH;    // [B][2]
    float *dY = Y + (size_t)B * MOUT;      // [B][2]
    float *dA = dY + (size_t)B * MOUT;     // [B][64]
    float *dB = dA + (size_t)B * MH;       // [B][64]
    float *lpart = dB + (size_t)B * MH;    // [nblk]
    float *cnt = lpart + B / MLP_T + 2;
    long long nblk = (B + MLP_T - 1) / MLP_T;
    note_launch();
    k_to_bf16<<<(MLP_NP + 255) / 256, 256>>>(m->w, m->wb, MLP_NP);
    note_launch();
    k_sum<<<1, 256>>>(mask, B * MOUT, cnt);
    note_launch();
    k_mlp_forward<<<(unsigned)nblk, MLP_T, fwd_smem()>>>(X, B, m->wb, m->norm, Y, Hs);
    note_launch();
    k_mlp_loss<<<(unsigned)nblk, MLP_T>>>(Y, T, mask, B, m->norm, cnt, dY, lpart);
    MCK(cudaMemset(m->g, 0, sizeof(float) * MLP_NP));
    const float *dZ = dY;
    float *bufs[2] = {dA, dB};
    for (int l = NLAYER - 1; l >= 0; --l) {
        const float *Ain = l == 0 ? X : Hs + (size_t)(l - 1) * B * MH;
        int lda = l == 0 ? MIN_ : MH;
        dim3 grid(dim_in(l) + 1, (unsigned)((B + GW_ROWS - 1) / GW_ROWS));
        note_launch();
        k_mlp_grad_w<<<grid, 64>>>(Ain, dim_in(l), lda, l == 0, m->norm, dZ, dim_out(l), B,
                                   m->g + off_w(l), m->g + off_b(l));
        if (l > 0) {
            float *dn = bufs[l & 1];
            note_launch();
            k_mlp_back_rows<<<(unsigned)nblk, MLP_T>>>(dZ, dim_out(l), m->wb + off_w(l),
                                                       Hs + (size_t)(l - 1) * B * MH, B, dn);
            dZ = dn;
        }
    }
    MCK(cudaGetLastError());
    std::vector<float> lp(nblk);
    MCK(cudaMemcpy(lp.data(), lpart, sizeof(float) * nblk, cudaMemcpyDeviceToHost));
    double s = 0.0;
    for (float v : lp) s += v;
    if (loss) *loss = (float)s;
    return CCFMM_OK;
}

extern "C" {

ccfmm_status ccfmm_mlp_create(ccfmm_mlp_t *out)
{
    if (!out) return mlp_fail(CCFMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    ccfmm_mlp_t m = new (std::nothrow) ccfmm_mlp_s();
    if (!m) return mlp_fail(CCFMM_ERR_ALLOC, "host allocation failed");
    cudaGetDevice(&m->device);
    cudaError_t e = cudaSuccess;
    float **fp[] = {&m->w, &m->g, &m->m1, &m->m2};
    for (float **q : fp)
        if (e == cudaSuccess) e = cudaMalloc(q, sizeof(float) * MLP_NP);
    if (e == cudaSuccess) e = cudaMalloc(&m->norm, sizeof(float) * NORM_N);
    if (e == cudaSuccess) e = cudaMalloc(&m->wb, sizeof(__nv_bfloat16) * MLP_NP);
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, sizeof(float) * MLP_NP);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, sizeof(float) * MLP_NP);
    if (e == cudaSuccess) e = cudaMemset(m->w, 0, sizeof(float) * MLP_NP);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ccfmm_mlp_destroy(m);
        return mlp_fail(CCFMM_ERR_ALLOC, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    std::vector<float> nrm(NORM_N, 0.f);
    for (int i = 0; i < MIN_; ++i) nrm[MIN_ + i] = 1.f;
    for (int i = 0; i < MOUT; ++i) nrm[2 * MIN_ + MOUT + i] = 1.f;
    cudaMemcpy(m->norm, nrm.data(), sizeof(float) * NORM_N, cudaMemcpyHostToDevice);
    *out = m;
    return CCFMM_OK;
}

void ccfmm_mlp_destroy(ccfmm_mlp_t m)
{
    if (!m) return;
    cudaFree(m->w);
    cudaFree(m->g);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->norm);
    cudaFree(m->wb);
    cudaFree(m->work);
    cudaGetLastError();
    delete m;
}

int32_t ccfmm_mlp_num_params(void) { return MLP_NP; }

ccfmm_status ccfmm_mlp_set_params(ccfmm_mlp_t m, const float *params, const float *norm)
{
    if (!m) return mlp_fail(CCFMM_ERR_ARG, "NULL handle");
    if (params) MCK(cudaMemcpy(m->w, params, sizeof(float) * MLP_NP, cudaMemcpyDefault));
    if (norm) MCK(cudaMemcpy(m->norm, norm, sizeof(float) * NORM_N, cudaMemcpyDefault));
    m->t = 0;
    MCK(cudaMemset(m->m1, 0, sizeof(float) * MLP_NP));
    MCK(cudaMemset(m->m2, 0, sizeof(float) * MLP_NP));
    return CCFMM_OK;
}

ccfmm_status ccfmm_mlp_get_params(ccfmm_mlp_t m, float *params, float *norm)
{
    if (!m) return mlp_fail(CCFMM_ERR_ARG, "NULL handle");
    if (params) MCK(cudaMemcpy(params, m->w, sizeof(float) * MLP_NP, cudaMemcpyDefault));
    if (norm) MCK(cudaMemcpy(norm, m->norm, sizeof(float) * NORM_N, cudaMemcpyDefault));
    return CCFMM_OK;
}

ccfmm_status ccfmm_mlp_fit_norm(ccfmm_mlp_t m, const float *X, const float *T, const float *mask,
                                int64_t B)
{
    if (!m || !X || !T || !mask || B < 1) return mlp_fail(CCFMM_ERR_ARG, "bad argument");
    FBuf x, t, k;
    ccfmm_status st;
    if ((st = fbuf(x, X, B * MIN_)) || (st = fbuf(t, T, B * MOUT)) || (st = fbuf(k, mask, B * MOUT)))
        return st;
    note_launch();
    k_fit_norm<<<1, 32>>>(x.p, t.p, k.p, B, m->norm);
    MCK(cudaGetLastError());
    MCK(cudaDeviceSynchronize());
    return CCFMM_OK;
}

ccfmm_status ccfmm_mlp_gradient(ccfmm_mlp_t m, const float *X, const float *T, const float *mask,
                                int64_t B, float *grad_out, float *loss_out)
{
    if (!m || !X || !T || !mask || B < 1) return mlp_fail(CCFMM_ERR_ARG, "bad argument");
    FBuf x, t, k;
    ccfmm_status st;
    if ((st = fbuf(x, X, B * MIN_)) || (st = fbuf(t, T, B * MOUT)) || (st = fbuf(k, mask, B * MOUT)))
        return st;
    if ((st = mlp_grad(m, x.p, t.p, k.p, B, loss_out))) return st;
    if (grad_out) MCK(cudaMemcpy(grad_out, m->g, sizeof(float) * MLP_NP, cudaMemcpyDefault));
    return CCFMM_OK;
}

ccfmm_status ccfmm_mlp_train(ccfmm_mlp_t m, const float *X, const float *T, const float *mask,
                             int64_t B, int64_t batch, int32_t epochs, float lr, uint64_t seed,
                             float *loss_out)
{
    if (!m || !X || !T || !mask || B < 1 || batch < 1 || epochs < 1)
        return mlp_fail(CCFMM_ERR_ARG, "bad argument");
    FBuf x, t, k;
    ccfmm_status st;
    if ((st = fbuf(x, X, B * MIN_)) || (st = fbuf(t, T, B * MOUT)) || (st = fbuf(k, mask, B * MOUT)))
        return st;
    // epochs over a fixed sequence of contiguous mini-batches (the caller
    // shuffles the rows once); Adam with bias correction
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float last = 0.f;
    (void)seed;
    for (int ep = 0; ep < epochs; ++ep) {
        double acc = 0.0;
        int nb = 0;
        for (long long r0 = 0; r0 < B; r0 += batch) {
            long long nbx = std::min<long long>(batch, B - r0);
            float l = 0.f;
            if ((st = mlp_grad(m, x.p + r0 * MIN_, t.p + r0 * MOUT, k.p + r0 * MOUT, nbx, &l)))
                return st;
            ++m->t;
            float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
            note_launch();
            k_adam<<<(MLP_NP + 255) / 256, 256>>>(m->w, m->g, m->m1, m->m2, MLP_NP, lr, b1, b2,
                                                 eps, c1, c2);
            acc += l;
            ++nb;
        }
        last = (float)(acc / std::max(nb, 1));
    }
    MCK(cudaGetLastError());
    MCK(cudaDeviceSynchronize());
    if (loss_out) *loss_out = last;
    return CCFMM_OK;
}

ccfmm_status ccfmm_mlp_predict(ccfmm_mlp_t m, const float *X, int64_t B, float *Y)
{
    if (!m || !X || !Y || B < 1) return mlp_fail(CCFMM_ERR_ARG, "bad argument");
    FBuf x;
    ccfmm_status st;
    if ((st = fbuf(x, X, B * MIN_))) return st;
    float *dy = nullptr;
    bool own = !dev_ptr(Y);
    if (own) MCK(cudaMalloc(&dy, sizeof(float) * B * MOUT));
    else dy = Y;
    long long nblk = (B + MLP_T - 1) / MLP_T;
    note_launch(3);
    k_to_bf16<<<(MLP_NP + 255) / 256, 256>>>(m->w, m->wb, MLP_NP);
    k_mlp_forward<<<(unsigned)nblk, MLP_T, fwd_smem()>>>(x.p, B, m->wb, m->norm, dy, nullptr);
    k_destandardise<<<(unsigned)((B * MOUT + 255) / 256), 256>>>(dy, B, m->norm);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && own) e = cudaMemcpy(Y, dy, sizeof(float) * B * MOUT, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (own) cudaFree(dy);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return mlp_fail(CCFMM_ERR_CUDA, cudaGetErrorString(e));
    }
    return CCFMM_OK;
}

// Nine features of a dipole set (positions N x 3 float64, host or device):
//  0 log10 N
//  1..3 occupancy of the depth-Lr cells of the bisection tree, Lr =
//       max(0, floor(log2(N/16))): slog(CV^2), slog(skewness),
//       slog(excess kurtosis), slog(x) = sign(x) log10(1 + |x|)
//  4 coefficient of variation of the nearest-neighbour distance (sample of
//    min(N, 2048) points)
//  5 min / mean of those distances
//  6 Clark-Evans ratio: mean distance / (0.55396 (V/N)^(1/3)), V = box volume
//  7, 8 box extents sorted: middle / largest, smallest / largest
ccfmm_status ccfmm_features(const double *positions, int64_t N, float *out9)
{
    if (!positions || !out9 || N < 2) return mlp_fail(CCFMM_ERR_ARG, "bad argument");
    double *dp = const_cast<double *>(positions);
    bool ownp = !dev_ptr(positions);
    std::vector<void *> frees;
    auto cleanup = [&]() {
        for (void *q : frees) cudaFree(q);
    };
#define FCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            cleanup();                                                                           \
            return mlp_fail(CCFMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
        }                                                                                        \
    } while (0)
    if (ownp) {
        FCK(cudaMalloc(&dp, sizeof(double) * 3 * N));
        frees.push_back(dp);
        FCK(cudaMemcpy(dp, positions, sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
    }
    double *box6, *partial, *mom4;
    int *flags, *cnt, *idx;
    uint32_t *keys;
    Geom *g;
    float4 *p4;
    float *nn;
    int Lr = 0;
    while (Lr < 20 && (double)N / (double)(1ll << (Lr + 1)) >= 16.0) ++Lr;
    long long ncell = 1ll << Lr;
    int S = (int)std::min<long long>(N, 2048);
    FCK(cudaMalloc(&box6, 6 * sizeof(double)));
    frees.push_back(box6);
    FCK(cudaMalloc(&partial, 6 * 1024 * sizeof(double)));
    frees.push_back(partial);
    FCK(cudaMalloc(&mom4, 4 * sizeof(double)));
    frees.push_back(mom4);
    FCK(cudaMalloc(&flags, sizeof(int)));
    frees.push_back(flags);
    FCK(cudaMalloc(&cnt, sizeof(int) * ncell));
    frees.push_back(cnt);
    FCK(cudaMalloc(&idx, sizeof(int) * N));
    frees.push_back(idx);
    FCK(cudaMalloc(&keys, sizeof(uint32_t) * N));
    frees.push_back(keys);
    FCK(cudaMalloc(&g, sizeof(Geom)));
    frees.push_back(g);
    FCK(cudaMalloc(&p4, sizeof(float4) * N));
    frees.push_back(p4);
    FCK(cudaMalloc(&nn, sizeof(float) * S));
    frees.push_back(nn);
    FCK(cudaMemset(flags, 0, sizeof(int)));
    FCK(cudaMemset(cnt, 0, sizeof(int) * ncell));
    FCK(cudaMemset(mom4, 0, 4 * sizeof(double)));
    launch_bbox(dp, N, nullptr, box6, partial, flags, 0);
    launch_geom(box6, g, 0);
    launch_keys(dp, N, g, keys, idx, flags, 0, 0);
    note_launch(4);
    k_cell_hist<<<(unsigned)((N + 255) / 256), 256>>>(keys, N, Lr, cnt);
    k_count_moments<<<(unsigned)std::min<long long>((ncell + 255) / 256, 1024), 256>>>(cnt, ncell, mom4);
    k_to_f32<<<(unsigned)((N + 255) / 256), 256>>>(dp, N, p4);
    k_nn_sample<<<(S + 127) / 128, 128>>>(p4, N, S, nn);
    FCK(cudaGetLastError());
    double hb[6], hm[4];
    int hf = 0;
    std::vector<float> hnn(S);
    FCK(cudaMemcpy(hb, box6, sizeof(hb), cudaMemcpyDeviceToHost));
    FCK(cudaMemcpy(hm, mom4, sizeof(hm), cudaMemcpyDeviceToHost));
    FCK(cudaMemcpy(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost));
    FCK(cudaMemcpy(hnn.data(), nn, sizeof(float) * S, cudaMemcpyDeviceToHost));
    cleanup();
#undef FCK
    if (hf & FLAG_NONFINITE) return mlp_fail(CCFMM_ERR_ARG, "non-finite position");
    // central moments of the counts from the raw sums
    double n = (double)ncell, m1 = hm[0] / n, m2 = hm[1] / n, m3 = hm[2] / n, m4 = hm[3] / n;
    double var = m2 - m1 * m1;
    double c3 = m3 - 3 * m1 * m2 + 2 * m1 * m1 * m1;
    double c4 = m4 - 4 * m1 * m3 + 6 * m1 * m1 * m2 - 3 * m1 * m1 * m1 * m1;
    double sd = var > 0 ? sqrt(var) : 0.0;
    double cv2 = m1 > 0 ? var / (m1 * m1) : 0.0;
    double skew = sd > 0 ? c3 / (sd * sd * sd) : 0.0;
    double kurt = sd > 0 ? c4 / (var * var) - 3.0 : 0.0;
    auto slog = [](double x) { return (x >= 0 ? 1.0 : -1.0) * log10(1.0 + fabs(x)); };
    double s1 = 0, s2 = 0, mn = INFINITY;
    for (float v : hnn) {
        s1 += v;
        s2 += (double)v * v;
        mn = std::min(mn, (double)v);
    }
    double mean = s1 / S, nsd = sqrt(std::max(s2 / S - mean * mean, 0.0));
    double ext[3] = {hb[3] - hb[0], hb[4] - hb[1], hb[5] - hb[2]};
    std::sort(ext, ext + 3);
    double vol = ext[0] * ext[1] * ext[2];
    double ce = vol > 0 ? mean / (0.55396 * cbrt(vol / (double)N)) : 0.0;
    float f[9] = {(float)log10((double)N), (float)slog(cv2), (float)slog(skew), (float)slog(kurt),
                  (float)(mean > 0 ? nsd / mean : 0.0), (float)(mean > 0 ? mn / mean : 0.0),
                  (float)ce, (float)(ext[1] / ext[2]), (float)(ext[0] / ext[2])};
    for (int i = 0; i < 9; ++i) out9[i] = f[i];
    return CCFMM_OK;
}


// The paper's rule of thumb: leaf occupancy by Eq. so; (p, alpha_m) =
// (5, 0.71) when about 1 % average error is enough, else (6, 0.48) (Sec. IV).
static void rule_of_thumb(double target, int *p, double *theta, double *leaf)
{
    if (target >= 1e-2) {
        *p = 5;
        *theta = 0.71;
    } else {
        *p = 6;
        *theta = 0.48;
    }
    *leaf = ccfmm_leaf_size_rule(*p);
}

ccfmm_status fmm_select(ccfmm_mlp_t m, const double *positions, int64_t N, double target_error,
                        int32_t *p_out, double *theta_out, double *leaf_out, int32_t *fallback_out)
{
    if (!positions || !p_out || !theta_out || !leaf_out || N < 2 || !(target_error > 0))
        return mlp_fail(CCFMM_ERR_ARG, "bad argument");
    int p;
    double th, lf;
    rule_of_thumb(target_error, &p, &th, &lf);
    int fb = 1;
    if (m) {
        float f9[9];
        ccfmm_status st = ccfmm_features(positions, N, f9);
        if (st != CCFMM_OK) return st;
        float nrm[NORM_N];
        if (cudaMemcpy(nrm, m->norm, sizeof(nrm), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return mlp_fail(CCFMM_ERR_CUDA, "reading the network's normalisation failed");
        }
        // inside the training range: every feature within 5 standard deviations
        bool inside = true;
        for (int i = 0; i < 9; ++i)
            if (fabsf((f9[i] - nrm[i]) / nrm[MIN_ + i]) > 5.f) inside = false;
        if (inside) {
            const int P[7] = {2, 3, 4, 5, 6, 7, 8};
            const double TH[5] = {0.3, 0.4, 0.5, 0.6, 0.7};
            const double LF[5] = {4, 8, 16, 32, 64};
            std::vector<float> X;
            for (int a = 0; a < 7; ++a)
                for (int b = 0; b < 5; ++b)
                    for (int c = 0; c < 5; ++c) {
                        for (int i = 0; i < 9; ++i) X.push_back(f9[i]);
                        X.push_back((float)P[a]);
                        X.push_back((float)TH[b]);
                        X.push_back((float)log2(LF[c]));
                    }
            std::vector<float> Y(175 * 2);
            st = ccfmm_mlp_predict(m, X.data(), 175, Y.data());
            if (st != CCFMM_OK) return st;
            // fastest configuration whose predicted error is below the target
            // with a factor-2 margin
            double lt = log10(target_error) - log10(2.0), best = INFINITY;
            for (int r = 0; r < 175; ++r)
                if (Y[2 * r + 1] <= lt && Y[2 * r] < best) {
                    best = Y[2 * r];
                    p = (int)X[12 * r + 9];
                    th = X[12 * r + 10];
                    lf = exp2((double)X[12 * r + 11]);
                    fb = 0;
                }
        }
    }
    *p_out = p;
    *theta_out = th;
    *leaf_out = lf;
    if (fallback_out) *fallback_out = fb;
    return CCFMM_OK;
}

}  // extern "C"
