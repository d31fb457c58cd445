// Two-scale coarse-graining (Section III-C; Algorithm 1, the first step of an iteration):
// the coarse design z_C holds the mean of z over each N_B x N_B x N_B block of elements.
// The last block along an axis that N_B does not divide holds the remaining elements.
// One thread per block; the block sum is accumulated in double (the kernel runs once per
// optimisation iteration and reads each element once).
#include "common.cuh"
#include "host.h"

namespace tomo {

template <typename T>
__global__ void k_coarse_grain(Geom g, int nb, int cx, int cy, int cz, const T* __restrict__ z,
                               T* __restrict__ zc) {
  PDL_ENTER();
  const int nc = cx * cy * cz;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nc; b += gridDim.x * blockDim.x) {
    const int I = b % cx, J = (b / cx) % cy, K = b / (cx * cy);
    const int i0 = I * nb, j0 = J * nb, k0 = K * nb;
    const int i1 = min(i0 + nb, g.nx), j1 = min(j0 + nb, g.ny), k1 = min(k0 + nb, g.nz);
    double s = 0.0;
    for (int k = k0; k < k1; ++k)
      for (int j = j0; j < j1; ++j) {
        const T* row = z + (size_t)g.nx * (j + (size_t)g.ny * k);
        for (int i = i0; i < i1; ++i) s += (double)row[i];
      }
    zc[b] = (T)(s / (double)((i1 - i0) * (j1 - j0) * (k1 - k0)));
  }
}

template <typename T>
cudaError_t launch_coarse_grain(cudaStream_t st, Geom g, int nb, const T* z, T* zc) {
  const int cx = (g.nx + nb - 1) / nb, cy = (g.ny + nb - 1) / nb, cz = (g.nz + nb - 1) / nb;
  const int nc = cx * cy * cz;
  int blocks = (nc + 127) / 128;
  if (blocks > 8192) blocks = 8192;
  return pdl_launch(k_coarse_grain<T>, blocks, 128, 0, st, g, nb, cx, cy, cz, z, zc);
}

template cudaError_t launch_coarse_grain<float>(cudaStream_t, Geom, int, const float*, float*);
template cudaError_t launch_coarse_grain<double>(cudaStream_t, Geom, int, const double*,
                                                 double*);

}  // namespace tomo
