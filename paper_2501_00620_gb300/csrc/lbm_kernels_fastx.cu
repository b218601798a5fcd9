// Launchers of the staged step kernel's FP32-only tiles (kFastOwn3,
// kFastOwn2): the force/MRT tiles and the walls tiles.
#include "lbm_fast_launch.cuh"

namespace lbm {

int n_own_variants(int D) {
    return D == 3 ? (int)(sizeof(kFastOwn3) / sizeof(kFastOwn3[0]))
                  : (D == 2 ? (int)(sizeof(kFastOwn2) / sizeof(kFastOwn2[0])) : 0);
}
Variant own_variant(int D, int k) {
    return D == 3 ? Variant{kFastOwn3[k].tx, kFastOwn3[k].ty} : Variant{kFastOwn2[k].tx, kFastOwn2[k].ty};
}
int own_kind(int D, int k) {
    const int pfb = D == 3 ? kFastOwn3[k].pfb : kFastOwn2[k].pfb;
    return (pfb & 16) ? 2 : ((pfb & 8) ? 1 : 0);
}

#define LBM_OWN_CASE(DD, TAB, K)                                                                      \
    case K:                                                                                           \
        if (box) {                                                                                    \
            fast_box<DD, float, TAB[K].tx, TAB[K].ty, TAB[K].pfb, TAB[K].mb>(box);                    \
            return cudaSuccess;                                                                       \
        }                                                                                             \
        return launch_fast<DD, float, TAB[K].tx, TAB[K].ty, TAB[K].pfb, TAB[K].mb, false>(*ta, st);

cudaError_t fast_own(int D, int k, const TmaArgs* ta, TmaBox* box, cudaStream_t st) {
    if (ta && (ta->s.fixed_x || ta->s.halo)) return cudaErrorInvalidValue;
    if (D == 3) {
        static_assert(sizeof(kFastOwn3) / sizeof(kFastOwn3[0]) == 2, "one case per tile");
        switch (k) {
            LBM_OWN_CASE(3, kFastOwn3, 0)
            LBM_OWN_CASE(3, kFastOwn3, 1)
            default: return cudaErrorInvalidValue;
        }
    }
    if (D == 2) {
        static_assert(sizeof(kFastOwn2) / sizeof(kFastOwn2[0]) == 2, "one case per tile");
        switch (k) {
            LBM_OWN_CASE(2, kFastOwn2, 0)
            LBM_OWN_CASE(2, kFastOwn2, 1)
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}
#undef LBM_OWN_CASE

}  // namespace lbm
