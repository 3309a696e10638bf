// prims.cu -- device-wide exclusive scan and stable LSD radix sort used by
// the tree build (key sort) and the list builders (CSR offsets).
#include "ccfmm_dev.cuh"

namespace ccfmm {

constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_B = SCAN_T * SCAN_I;

// exclusive block scan of one value per thread; *total gets the block sum
__device__ __forceinline__ int block_exclusive_scan(int v, int *sm, int *total)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < nw ? sm[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sm[lane] = s;
    }
    __syncthreads();
    int prefix = warp ? sm[warp - 1] : 0;
    *total = sm[nw - 1];
    __syncthreads();
    return prefix + x - v;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(const int *in, int *out, long long n,
                                                        int *bsum, int *total)
{
    __shared__ int sm[32];
    long long base = (long long)blockIdx.x * SCAN_B + (long long)threadIdx.x * SCAN_I;
    int v[SCAN_I];
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        long long j = base + i;
        v[i] = j < n ? in[j] : 0;
        s += v[i];
    }
    int tot;
    int ex = block_exclusive_scan(s, sm, &tot);
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        long long j = base + i;
        if (j < n) out[j] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = tot;
        if (gridDim.x == 1 && total) *total = tot;
    }
}

__global__ void k_scan_add(int *out, long long n, const int *boff)
{
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] += boff[j / SCAN_B];
}

size_t scan_temp_bytes(long long n)
{
    size_t b = 0;
    long long m = n;
    do {
        m = (m + SCAN_B - 1) / SCAN_B;
        b += (size_t)m * sizeof(int) + 256;
    } while (m > 1);
    return b;
}

void scan_exclusive(const int *in, int *out, long long n, int *d_total, void *temp, cudaStream_t s)
{
    if (n <= 0) {
        if (d_total) cudaMemsetAsync(d_total, 0, sizeof(int), s);
        return;
    }
    long long nb = (n + SCAN_B - 1) / SCAN_B;
    int *bsum = (int *)temp;
    char *next = (char *)temp + (((size_t)nb * sizeof(int) + 255) / 256) * 256;
    note_launch();
    k_scan_blocks<<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, n, bsum, d_total);
    if (nb > 1) {
        scan_exclusive(bsum, bsum, nb, d_total, next, s);
        note_launch();
        k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, bsum);
    }
}

// Two arrays of the same length in one launch set (blockIdx.y picks the
// array): the near and far counts of a level.
struct Scan2 {
    const int *in[2];
    int *out[2];
    int *total[2];
};

__global__ void __launch_bounds__(SCAN_T) k_scan_blocks2(Scan2 a, long long n, int *bsum,
                                                         long long nb)
{
    __shared__ int sm[32];
    const int y = blockIdx.y;
    const int *in = a.in[y];
    int *out = a.out[y];
    long long base = (long long)blockIdx.x * SCAN_B + (long long)threadIdx.x * SCAN_I;
    int v[SCAN_I];
    int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        long long j = base + i;
        v[i] = j < n ? in[j] : 0;
        s += v[i];
    }
    int tot;
    int ex = block_exclusive_scan(s, sm, &tot);
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        long long j = base + i;
        if (j < n) out[j] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) {
        bsum[y * nb + blockIdx.x] = tot;
        if (gridDim.x == 1 && a.total[y]) *a.total[y] = tot;
    }
}

__global__ void k_scan_add2(int *out0, int *out1, long long n, const int *boff, long long nb)
{
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (blockIdx.y == 0)
        out0[j] += boff[j / SCAN_B];
    else
        out1[j] += boff[nb + j / SCAN_B];
}

void scan_exclusive2(const int *in0, int *out0, int *total0, const int *in1, int *out1,
                     int *total1, long long n, void *temp, cudaStream_t s)
{
    if (n <= 0) {
        if (total0) cudaMemsetAsync(total0, 0, sizeof(int), s);
        if (total1) cudaMemsetAsync(total1, 0, sizeof(int), s);
        return;
    }
    long long nb = (n + SCAN_B - 1) / SCAN_B;
    int *bsum = (int *)temp;  // [2][nb]
    char *next = (char *)temp + (((size_t)2 * nb * sizeof(int) + 255) / 256) * 256;
    Scan2 a;
    a.in[0] = in0;
    a.in[1] = in1;
    a.out[0] = out0;
    a.out[1] = out1;
    a.total[0] = total0;
    a.total[1] = total1;
    note_launch();
    k_scan_blocks2<<<dim3((unsigned)nb, 2), SCAN_T, 0, s>>>(a, n, bsum, nb);
    if (nb > 1) {
        scan_exclusive2(bsum, bsum, total0, bsum + nb, bsum + nb, total1, nb, next, s);
        note_launch();
        k_scan_add2<<<dim3((unsigned)((n + 255) / 256), 2), 256, 0, s>>>(out0, out1, n, bsum, nb);
    }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits, tiles of 2048 keys (8 rounds of 256).
// Within a tile the rank of a key among equal digits follows input order:
// rounds in order, warps in order inside a round, lanes in order in a warp.
// ---------------------------------------------------------------------------
constexpr int RS_T = 256, RS_R = 8, RS_TILE = RS_T * RS_R;

__global__ void __launch_bounds__(RS_T) k_radix_count(const uint32_t *keys, long long n, int shift,
                                                      int *counts, int ntiles)
{
    __shared__ int hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_R; ++r) {
        long long i = base + r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&hist[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(long long)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

__global__ void __launch_bounds__(RS_T) k_radix_scatter(const uint32_t *kin, const int *vin,
                                                        uint32_t *kout, int *vout, long long n,
                                                        int shift, const int *offs, int ntiles)
{
    __shared__ int wcnt[RS_T / 32][256];
    __shared__ int base[256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    base[tid] = offs[(long long)tid * ntiles + blockIdx.x];
    for (int r = 0; r < RS_R; ++r) {
        for (int i = tid; i < (RS_T / 32) * 256; i += RS_T) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        long long idx = (long long)blockIdx.x * RS_TILE + r * RS_T + tid;
        bool valid = idx < n;
        uint32_t key = valid ? kin[idx] : 0u;
        int d = valid ? (int)((key >> shift) & 255u) : -1;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & ((1u << lane) - 1u));
        int leader = 31 - __clz(peers);
        if (valid && lane == leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        int run = 0;
#pragma unroll
        for (int w = 0; w < RS_T / 32; ++w) {
            int c = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            int pos = base[d] + wcnt[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = vin[idx];
        }
        __syncthreads();
        base[tid] += run;
        __syncthreads();
    }
}

size_t radix_temp_bytes(long long n)
{
    long long ntiles = (n + RS_TILE - 1) / RS_TILE;
    size_t cnt = (size_t)ntiles * 256;
    return ((cnt * sizeof(int) + 255) / 256) * 256 + scan_temp_bytes((long long)cnt);
}

void radix_sort(const uint32_t *k_in, const int *v_in, uint32_t *k_out, int *v_out,
                uint32_t *k_tmp, int *v_tmp, long long n, int bits, void *temp, cudaStream_t s)
{
    if (n <= 0) return;
    int passes = (bits + 7) / 8;
    if (passes == 0) {
        cudaMemcpyAsync(k_out, k_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(v_out, v_in, n * sizeof(int), cudaMemcpyDeviceToDevice, s);
        return;
    }
    long long ntiles = (n + RS_TILE - 1) / RS_TILE;
    int *counts = (int *)temp;
    void *stemp = (char *)temp + (((size_t)ntiles * 256 * sizeof(int) + 255) / 256) * 256;
    const uint32_t *ki = k_in;
    const int *vi = v_in;
    for (int ps = 0; ps < passes; ++ps) {
        // land the last pass in (k_out, v_out)
        bool to_out = ((passes - 1 - ps) % 2) == 0;
        uint32_t *ko = to_out ? k_out : k_tmp;
        int *vo = to_out ? v_out : v_tmp;
        note_launch();
        k_radix_count<<<(unsigned)ntiles, RS_T, 0, s>>>(ki, n, 8 * ps, counts, (int)ntiles);
        scan_exclusive(counts, counts, ntiles * 256, nullptr, stemp, s);
        note_launch();
        k_radix_scatter<<<(unsigned)ntiles, RS_T, 0, s>>>(ki, vi, ko, vo, n, 8 * ps, counts,
                                                          (int)ntiles);
        ki = ko;
        vi = vo;
    }
}

}  // namespace ccfmm
