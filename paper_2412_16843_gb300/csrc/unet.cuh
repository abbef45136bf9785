// Learned first guess of the pressure solve: a 3D U-Net (4 levels, 16..128
// channels, 726,993 parameters) whose convolutions run on the tensor cores in
// BF16 with FP32 accumulation.  The paper has no network; this is a form of
// the solver.  Declarations shared by unet.cu and cdi_api.cu.
#pragma once

#include "cdi_internal.cuh"

struct cdi_unet;

namespace cdi {

// First guess p0 of div(grad p / rho) = f on a grid whose extents are the
// network's: input (f / rms(f), rho / max(rho1, rho2)) in BF16, output scaled
// by rms(f) max(rho) h^2 (h: the grid spacing).  fnorm_dev holds ||f||_2
// (device scalar).
template <typename T>
cudaError_t unet_predict_device(cdi_unet* net, const double* f_dev, const T* phi_dev, double rho1, double rho2,
                                const double* fnorm_dev, double h, double* p_dev, cudaStream_t s);

// the network's grid extents (nx, ny, nz)
void unet_extents(const cdi_unet* net, int* n);

}  // namespace cdi
