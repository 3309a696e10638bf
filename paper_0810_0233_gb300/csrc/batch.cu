// batch.cu -- ensemble time step: every moment of every sample is turned
// about a random axis by a random angle (a project addition; the paper has
// no time stepping).  Random numbers: Philox4x64-10 (Salmon, Moraes, Dror,
// Shaw, SC 2011) with key (seed, step) and counter (global dipole index, 0,
// 0, 0); u_i = (x_i >> 11) 2^-53; axis z = 1 - 2 u0, phi = 2 pi u1; angle =
// max_angle u2; Rodrigues' formula m' = m cos a + (k x m) sin a +
// k (k.m)(1 - cos a), in FP64.
#include "ccfmm_dev.cuh"
#include "stages.cuh"

namespace ccfmm {

__global__ void k_rotate(double *mom, long long n, const RotateParams *prm)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rotate_one(mom, i, prm);
}

void launch_rotate(double *mom, long long n, const RotateParams *prm, cudaStream_t s)
{
    if (n <= 0) return;
    note_launch();
    k_rotate<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mom, n, prm);
}

}  // namespace ccfmm
