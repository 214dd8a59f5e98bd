// cnn_layout.cuh -- layouts shared by the learned proposal's forward
// (cnn.cu) and backward (cnn_bwd.cu) kernels: the fp32 master parameter
// vector and the per-patch record of saved activations.
#pragma once

#include "vs_common.cuh"

namespace vs {
namespace cnn {

constexpr int kPatch = 65;

// ---- master parameter layout (fp32): w_l [32][cin][3][3], b_l [32], fw [32], fb
constexpr int kNParams = 288 + 32 + 4 * (9216 + 32) + 33;
__host__ __device__ constexpr int off_w(int l) { return l == 0 ? 0 : 320 + (l - 1) * 9248; }
__host__ __device__ constexpr int off_b(int l) { return l == 0 ? 288 : 320 + (l - 1) * 9248 + 9216; }
constexpr int kOffFw = 320 + 4 * 9248;

// ---- activations saved for the backward pass, per patch (bytes)
constexpr int kA1 = 33 * 33 * 32 * 2, kA2 = 17 * 17 * 32 * 2, kA3 = 9 * 9 * 32 * 2,
              kA4 = 5 * 5 * 32 * 2, kA5 = 5 * 5 * 32 * 2;
constexpr int kSvA1 = 0, kSvA2 = kSvA1 + kA1, kSvA3 = kSvA2 + kA2, kSvA4 = kSvA3 + kA3,
              kSvA5 = kSvA4 + kA4, kSvHead = kSvA5 + kA5;  // head: g[32], logit, y (fp32)
constexpr int kSaveBytes = ((kSvHead + 34 * 4) + 127) & ~127;
constexpr int kSvInput = kSaveBytes;                       // x0: 65x65 bf16
constexpr int kSaveBytesTotal = kSaveBytes + ((kPatch * kPatch * 2 + 127) & ~127);

// geometry of conv layer l (0-based): input / output side, channels, stride,
// and where its input and output sit in a save record
struct LayerGeo {
    int Hin, Win, Cin, Hout, Wout, stride;
    int sv_in, sv_out;  // byte offsets of the layer's input / output in a save record
};

__host__ __device__ inline LayerGeo layer_geo(int l) {
    LayerGeo g;
    g.Hin = g.Win = l == 0 ? 65 : l == 1 ? 33 : l == 2 ? 17 : l == 3 ? 9 : 5;
    g.Hout = g.Wout = l == 0 ? 33 : l == 1 ? 17 : l == 2 ? 9 : 5;
    g.Cin = l == 0 ? 1 : 32;
    g.stride = l == 4 ? 1 : 2;
    g.sv_in = l == 0 ? kSvInput : l == 1 ? kSvA1 : l == 2 ? kSvA2 : l == 3 ? kSvA3 : kSvA4;
    g.sv_out = l == 0 ? kSvA1 : l == 1 ? kSvA2 : l == 2 ? kSvA3 : l == 3 ? kSvA4 : kSvA5;
    return g;
}

}  // namespace cnn
}  // namespace vs
