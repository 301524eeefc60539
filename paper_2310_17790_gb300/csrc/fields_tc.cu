// BF16 field networks on the tcgen05 tensor cores (precision NSF_PREC_BF16).
// (Packing helpers; the kernels follow.)
#include "device_common.cuh"

namespace nsf {

// Hidden-layer operand order: the K-major, no-swizzle "core matrix" layout of
// tcgen05 shared-memory descriptors.  A core matrix is 8 rows x 16 bytes
// (8 bf16 along K) stored contiguously (128 B).  For a [N = width][K = width]
// weight matrix (row = output unit n, column = input unit k) the core matrix
// (n / 8, k / 8) is stored at ((k / 8) * (width / 8) + n / 8) * 64 elements, so
// that the 8-row groups along N are adjacent (stride 128 B) and successive
// K groups are width * 16 bytes apart.
size_t tc_pack_size(int width) { return (size_t)width * width; }

void tc_pack_layer(const float *W, int width, __nv_bfloat16 *dst) {
    const int g = width / 8;
    for (int n = 0; n < width; ++n)
        for (int k = 0; k < width; ++k) {
            size_t core = (size_t)(k / 8) * g + (n / 8);
            size_t idx = core * 64 + (n % 8) * 8 + (k % 8);
            dst[idx] = __float2bfloat16_rn(W[(size_t)n * width + k]);
        }
}

int jac_grid_size_tc(const FieldsDev &fd, int n) { return 1; }

cudaError_t launch_fields_tc(const FieldsDev &, const float *, int, int, int,
                             const FieldJob *, int *, cudaStream_t) {
    return cudaErrorNotSupported;
}

cudaError_t launch_jacobian_tc(const FieldsDev &, const float *, int, int,
                               const double *, float *, float *, const GnArgs *,
                               int *, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace nsf
