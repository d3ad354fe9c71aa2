// Instantiations of the lattice kernels for the moment-space collision of
// Sec. 2 (relaxation times: shear and bulk modes tau, momentum and
// non-hydrodynamic modes 1; templates in lbm_impl.cuh).
#include "lbm_impl.cuh"

namespace vefd {

cudaError_t launch_lattice_mrt(int lattice, int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s,
                               const void* tensor_map, int rev, int tile, Parts parts) {
    return launch_lattice_coll<1>(lattice, ncomp, p, b, s, tensor_map, rev, tile, parts);
}

cudaError_t launch_lattice_zm_mrt(int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s,
                                  const void* tensor_map, int zs, int rev) {
    return launch_zm_coll<1>(ncomp, p, b, s, tensor_map, zs, rev);
}

cudaError_t launch_lattice_batch_mrt(int ncomp, int prec, int tile, const EnsMember* members, const int* start,
                                     int nm, int items, int parity, bool pdl, cudaStream_t s) {
    return launch_lattice_batch_coll<1>(ncomp, prec, tile, members, start, nm, items, parity, pdl, s);
}

}  // namespace vefd
