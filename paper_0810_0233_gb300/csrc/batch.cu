// batch.cu -- ensemble time step: every moment of every sample is turned
// about a random axis by a random angle (a project addition; the paper has
// no time stepping).  Random numbers: Philox4x64-10 (Salmon, Moraes, Dror,
// Shaw, SC 2011) with key (seed, step) and counter (global dipole index, 0,
// 0, 0); u_i = (x_i >> 11) 2^-53; axis z = 1 - 2 u0, phi = 2 pi u1; angle =
// max_angle u2; Rodrigues' formula m' = m cos a + (k x m) sin a +
// k (k.m)(1 - cos a), in FP64.
#include "ccfmm_dev.cuh"

namespace ccfmm {

__device__ __forceinline__ void philox4x64(unsigned long long c[4], unsigned long long k0,
                                           unsigned long long k1)
{
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

__global__ void k_rotate(double *mom, long long n, const RotateParams *prm)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double two53 = 1.0 / 9007199254740992.0;
    unsigned long long x[4] = {(unsigned long long)i, 0ull, 0ull, 0ull};
    philox4x64(x, prm->seed, prm->step);
    double u0 = (double)(x[0] >> 11) * two53, u1 = (double)(x[1] >> 11) * two53;
    double u2 = (double)(x[2] >> 11) * two53;
    // phi = 2 pi u1 by sincospi(2 u1) (no argument reduction by pi), the
    // angle's sine and cosine from one sincos
    double z = 1.0 - 2.0 * u0, s = sqrt(1.0 - z * z), sp, cp;
    sincospi(2.0 * u1, &sp, &cp);
    double k[3] = {s * cp, s * sp, z};
    double a = prm->max_angle * u2, ca, sa;
    sincos(a, &sa, &ca);
    double m[3] = {mom[3 * i], mom[3 * i + 1], mom[3 * i + 2]};
    double kxm[3] = {k[1] * m[2] - k[2] * m[1], k[2] * m[0] - k[0] * m[2], k[0] * m[1] - k[1] * m[0]};
    double km = k[0] * m[0] + k[1] * m[1] + k[2] * m[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) mom[3 * i + d] = m[d] * ca + kxm[d] * sa + k[d] * km * (1.0 - ca);
}

void launch_rotate(double *mom, long long n, const RotateParams *prm, cudaStream_t s)
{
    if (n <= 0) return;
    note_launch();
    k_rotate<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mom, n, prm);
}

}  // namespace ccfmm
