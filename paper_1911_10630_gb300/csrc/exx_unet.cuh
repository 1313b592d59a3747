// exx_unet.cuh -- the learned CG warm start: a 3D U-Net (BF16 activations and
// weights, FP32 accumulation) and its host-side driver, shared by the guess
// C ABI (exx_unet.cu) and the solver's warm_start = 2 path (exx_api.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "exx_internal.h"

namespace exx {
namespace unet {

// Layer table: 3x3x3 convolutions with zero padding, ReLU after each one but
// the 1x1x1 head. Order = order of the flat parameter vector (W[27][cin][cout]
// then bias[cout] per layer; the head has w[16] then b[1]).
constexpr int kLayers = 15;
// input channels: rho / s on the PE ball, the multipole boundary values
// v_ME / (s delta^2) on the cube outside the ball, the ball mask
constexpr int kIn = 3;
constexpr int kMaskChannel = 2;
constexpr int kCin[kLayers] = {kIn, 16, 16, 32, 32, 64, 64, 128, 192, 64, 96, 32, 48, 16, 16};
constexpr int kCout[kLayers] = {16, 16, 32, 32, 64, 64, 128, 128, 64, 64, 32, 32, 16, 16, 1};
constexpr int kHead = 14;

size_t param_count();
size_t param_offset(int layer);  // offset of layer's W in the flat vector (bias follows W)

struct Net {
    int S = 0;          // input cube side (multiple of 8)
    int Bmax = 0;       // samples per call
    int n_sm = 0;
    size_t nparam = 0;
    float* params = nullptr;       // device FP32 master parameters
    float* grads = nullptr;        // device FP32 gradients
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* wfwd[kLayers] = {};  // packed BF16 weights (forward), layers 1..13
    __nv_bfloat16* wbwd[kLayers] = {};  // packed BF16 flipped/transposed weights (data gradient)
    int adam_t = 0;
    bool packed = false;
    // activations (BF16, channels last) and their gradients, sized for Bmax
    std::vector<void*> bufs;
    __nv_bfloat16 *x0a, *x0, *p0, *x1a, *x1, *p1, *x2a, *x2, *p2, *x3a, *x3;
    __nv_bfloat16 *c2, *y2a, *y2, *c1, *y1a, *y1, *c0, *y0a, *y0;
    __nv_bfloat16 *g_y0, *g_y0a, *g_c0, *g_y1, *g_y1a, *g_c1, *g_y2, *g_y2a, *g_c2;
    __nv_bfloat16 *g_x3, *g_x3a, *g_p2, *g_x2, *g_x2a, *g_p1, *g_x1, *g_x1a, *g_p0, *g_x0, *g_x0a;
    float* out = nullptr;           // [Bmax][S^3] FP32 network output
    float* gpart = nullptr;         // per-block / per-split partial sums of the gradient reductions
    float* d_loss = nullptr;        // [1]
    int* d_err = nullptr;           // tensor-core wait time-out flag
};

// All return cudaSuccess or the first CUDA error; time-outs of the tensor-core
// waits surface as cudaErrorLaunchTimeout from check_error().
cudaError_t create(Net& n, int S, int Bmax);
void destroy(Net& n);
cudaError_t pack(Net& n, cudaStream_t st);                       // params -> BF16 packed weights
cudaError_t forward(Net& n, const float* in, int B, cudaStream_t st);   // in: [B][S^3][kIn]; result in n.out
cudaError_t backward(Net& n, const float* in, const float* target, int B, cudaStream_t st);  // grads, loss
cudaError_t adam_step(Net& n, float lr, cudaStream_t st);
cudaError_t check_error(Net& n, cudaStream_t st);

// One 3x3x3 convolution on the tensor cores (exposed for its parity test).
// x [B][D][H][W][cin] BF16, wp packed by pack_weights, y [B][D][H][W][cout].
// epi 0: y = acc (+ bias); 1: ReLU(acc + bias); 2: acc * (mask > 0).
cudaError_t conv3_tc(const __nv_bfloat16* x, const __nv_bfloat16* wp, const float* bias,
                     const __nv_bfloat16* mask, __nv_bfloat16* y, int B, int D, int H, int W, int cin,
                     int cout, int epi, int* err, int n_sm, cudaStream_t st);
// w [27][cin][cout] FP32 -> packed BF16 operand of conv3_tc. flip = 1 packs the
// weights of the data gradient (a convolution from cout to cin channels with
// the taps mirrored).
cudaError_t pack_weights(const float* w, __nv_bfloat16* wp, int cin, int cout, int flip, cudaStream_t st);

// Network inputs of pairs k0 .. k0 + nk - 1 of the list: cube of side S
// centred on g_ij (offset o = index - S/2), channel 0 = rho / s on the PE
// ball, channel 1 = the multipole boundary values v_ME / (s d2) on the cube
// outside the ball (Eqs. mepole, me; l <= lmax), channel 2 = ball mask, s =
// max |rho| on the ball (scale[k - k0]). With vcache (the pairs' PE-ball
// potentials, FP32, list order), target receives v / (s d2) on the ball and 0
// elsewhere. input [nk][S^3][kIn], target [nk][S^3]. phi holds ostride values
// per orbital: full grids (box_org NULL) or compact boxes (as SolveParams).
cudaError_t sample_prep(const double* phi, const int N[3], const PairRec* pairs, int k0, int nk, int S,
                        const BallGeo& G, float* input, float* scale, float* target, const float* vcache, double d2,
                        const double delta[3], double dV, int lmax, const int* box_org, const int bdim[3],
                        long long ostride, cudaStream_t st);
// The multipole constants of the boundary channel (this unit's copy).
cudaError_t set_multipole_const_unet(const MultipoleConst& mc);
// vguess[k][p] = out[k - k0][cube(o_p)] * scale[k - k0] * d2 on the PE points
// p of pairs k0 .. k0 + nk - 1 (0 where o_p falls outside the cube).
cudaError_t guess_scatter(const float* out, const float* scale, int k0, int nk, int S, const BallGeo& G, double d2,
                          float* vguess, cudaStream_t st);

}  // namespace unet
}  // namespace exx
