// rbl_force_ewald.cu -- the force kernel with the LJ plus Ewald real-space pair,
// u(r) = 4 (r^-12 - r^-6) + q_i q_j erfc(alpha r) / r: the RBL applied unchanged to
// the short-range part of the Coulomb interaction (Sec. 2, closing remarks;
// Sec. 4).  Same core sum, batch, scale and reductions as the LJ kernel; its own
// translation unit so that both compile in parallel.
#include "rbl_force_kernel.cuh"

namespace rbl {

cudaError_t launch_force_kernel_ewald(const View &v, int step_offset, bool energy, cudaStream_t s, bool prepare)
{
    return launch_force_dispatch<true>(v, step_offset, energy, s, prepare);
}

cudaError_t launch_exact_energy_kernel_ewald(const View &v, cudaStream_t s)
{
    return launch_exact_dispatch<true>(v, s);
}

} // namespace rbl
