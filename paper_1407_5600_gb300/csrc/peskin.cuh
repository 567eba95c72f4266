// Three-point Peskin kernel weights for the blob-grid coupling (Eq. delta).
#pragma once

#include <cuda_runtime.h>

namespace mbk {

// For a blob at fractional node coordinate x (x = q/h - shift, shift = 0 along the component's
// own axis and 1/2 across it on the MAC grid), the only nodes with non-zero weight are the
// nearest node i0 = floor(x + 1/2) and its two neighbours.  With t = x - i0 in [-1/2, 1/2) and
// s = sqrt(1 - 3 t^2), the Roma-Peskin-Berger function gives
//   Phi at i0 - 1 = (2 - 3t - s)/6,  Phi at i0 = (1 + s)/3,  Phi at i0 + 1 = (2 + 3t - s)/6,
// which sum to 1, have zero first moment and squares summing to 1/2 for every t.
// The offset is taken in FP64 (positions are FP64); the weights in R.
// Returns i0 - 1, the index of the first node of the window.
template <typename R>
__device__ __forceinline__ int peskin_window(double x, R w[3])
{
    const double fl = floor(x + 0.5);
    const R t = static_cast<R>(x - fl);
    const R s = sqrt(R(1) - R(3) * t * t);
    w[0] = (R(2) - R(3) * t - s) * R(1.0 / 6.0);
    w[1] = (R(1) + s) * R(1.0 / 3.0);
    w[2] = (R(2) + R(3) * t - s) * R(1.0 / 6.0);
    return static_cast<int>(fl) - 1;
}

// MAC node offset of component `comp` along dimension `dim`, in mesh units.
__device__ __forceinline__ double mac_shift(int comp, int dim) { return comp == dim ? 0.0 : 0.5; }

// Periodic wrap of a position after a displacement smaller than the box.
__device__ __forceinline__ double wrap_position(double x, double L)
{
    if (x < 0.0) {
        x += L;
        if (x >= L) x -= L;
    } else if (x >= L) {
        x -= L;
    }
    return x;
}

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

}  // namespace mbk
