// Specializations of the multi-system energy kernel (multi_kernel.cuh) for
// the common compositions of a launch: systems of one dimension with
// uniform charges whose pair loops take at most two candidate slot counts.
#include "multi_kernel.cuh"

namespace ewald {

template <int DIM, int A, int B>
static MultiFn pick() {
    return k_multi_energy_t<float, DIM, (A < B ? A : B), (A < B ? B : A), false>;
}

MultiFn multi_kernel_spec(int dim, int a, int b) {
    if (a > b) std::swap(a, b);
    if (dim == 3) {
        // slot counts 0 (chunked lists), 4, 6, 8
        if (a == 0 && b == 0) return pick<3, 0, 0>();
        if (a == 0 && b == 4) return pick<3, 0, 4>();
        if (a == 0 && b == 6) return pick<3, 0, 6>();
        if (a == 0 && b == 8) return pick<3, 0, 8>();
        if (a == 4 && b == 4) return pick<3, 4, 4>();
        if (a == 4 && b == 6) return pick<3, 4, 6>();
        if (a == 4 && b == 8) return pick<3, 4, 8>();
        if (a == 6 && b == 6) return pick<3, 6, 6>();
        if (a == 6 && b == 8) return pick<3, 6, 8>();
        if (a == 8 && b == 8) return pick<3, 8, 8>();
    } else if (dim == 2) {
        if (a == 2 && b == 2) return pick<2, 2, 2>();
        if (a == 2 && b == 4) return pick<2, 2, 4>();
        if (a == 4 && b == 4) return pick<2, 4, 4>();
    }
    return nullptr;
}

}  // namespace ewald
