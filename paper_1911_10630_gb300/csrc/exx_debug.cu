// exx_debug.cu -- one application of the multigrid preconditioner, for tests.
//
// exx_apply_preconditioner runs one FP64 V-cycle (the stages of exx_mg.cuh
// that precondition the CG) on the context's largest PE ball in workspace
// slot 0, on one CTA, and returns z = M r on the ball. Tests check what makes
// the PCG a CG: M symmetric and positive definite, and close to A^-1.
#include <cuda_runtime.h>

#include "exx_mg.cuh"

namespace exx {

template <int NT>
__global__ void __launch_bounds__(NT) mg_apply_kernel(const __grid_constant__ SolveParams P, int geo,
                                                      const double* __restrict__ r, double* __restrict__ z) {
    const BallGeo G = P.geos[geo];
    const MGGeo& M = P.mg[geo];
    if (M.L < 1) return;  // no coarser level: the host refuses such a ball
    char* slot = P.ws;
    mg_vcycle<NT, double, 2>(P, G, M, slot, r);  // z in the level-0 Tc cube
    __syncthreads();
    const double* Tc = reinterpret_cast<const double*>(slot + P.off_tc);
    for (int k = threadIdx.x; k < G.n_pe; k += NT) z[k] = Tc[G.pt_cube[k]];
}

cudaError_t launch_mg_apply(const SolveParams& P, int geo, const double* r, double* z, cudaStream_t st) {
    mg_apply_kernel<256><<<1, 256, 0, st>>>(P, geo, r, z);
    return cudaGetLastError();
}

}  // namespace exx
