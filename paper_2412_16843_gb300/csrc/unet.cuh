// Learned first guess of the pressure solve: a 3D U-Net (4 levels, 16..128
// channels, 726,993 parameters) whose convolutions run on the tensor cores in
// BF16 with FP32 accumulation.  The paper has no network; this is a form of
// the solver.  Declarations shared by unet.cu and cdi_api.cu.
#pragma once

#include "cdi_internal.cuh"

struct cdi_unet;

namespace cdi {

// First guess p0 of div(grad p / rho) = f, written into the level-0 pressure
// of mg, on a grid whose extents are the network's: input (f / rms(f),
// rho / max(rho1, rho2)) in BF16, output scaled by rms(f) max(rho) h^2 (h:
// the grid spacing).  Reads f, its norm (S_FNORM) and, in the FP32-mixed
// form, its double-float mean from mg.
template <typename T>
cudaError_t unet_predict_device(cdi_unet* net, const MG& mg, const T* phi_dev, double rho1, double rho2, double h,
                                cudaStream_t s);

// the network's grid extents (nx, ny, nz)
void unet_extents(const cdi_unet* net, int* n);

}  // namespace cdi
