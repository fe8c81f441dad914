// fam_inst.cu -- kernel instantiation unit.  Compiled once per
// configuration with -DFAM_D=<1|2> -DFAM_P=<64|32> -DFAM_K=<3..6>; defines
// fam_pick_d<D>_p<P>_k<K>(), which binds the handle's launch table to the
// stage / OE / speed kernels of that configuration for the handle's equation.
#include "fam_internal.cuh"

#ifndef FAM_D
#error "FAM_D must be defined"
#endif

#if FAM_P == 64
typedef double Real;
#else
typedef float Real;
#endif

#define FAM_CAT_(a, b, c, d, e, f) a##b##c##d##e##f
#define FAM_CAT(a, b, c, d, e, f) FAM_CAT_(a, b, c, d, e, f)
#define FAM_PICK_NAME FAM_CAT(fam_pick_d, FAM_D, _p, FAM_P, _k, FAM_K)

bool FAM_PICK_NAME(fam_handle* h) {
  constexpr int K = FAM_K;
#if FAM_D == 1
  switch (h->eq) {
    case FAM_ADVECTION: h->ops = ops_of<Impl1D<Real, K, Advection1D<Real>>>(); return true;
    case FAM_BURGERS: h->ops = ops_of<Impl1D<Real, K, Burgers1D<Real>>>(); return true;
    case FAM_EULER: h->ops = ops_of<Impl1D<Real, K, Euler1D<Real>>>(); return true;
    case FAM_BUCKLEY: h->ops = ops_of<Impl1D<Real, K, BuckleyLeverett1D<Real>>>(); return true;
  }
#else
#define FAM_PICK2D(TXv, TYv)                                                                           \
  switch (h->eq) {                                                                                      \
    case FAM_ADVECTION: h->ops = ops_of2d<Impl2D<Real, K, Advection2D<Real>, TXv, TYv>>(); return true; \
    case FAM_BURGERS: h->ops = ops_of2d<Impl2D<Real, K, Burgers2D<Real>, TXv, TYv>>(); return true;     \
    case FAM_EULER: h->ops = ops_of2d<Impl2D<Real, K, Euler2D<Real>, TXv, TYv>>(); return true;         \
  }
  if (h->tile2d == 1) { FAM_PICK2D(32, 4) }
  else if (h->tile2d == 2) { FAM_PICK2D(16, 8) }
  else { FAM_PICK2D(32, 8) }
#undef FAM_PICK2D
#endif
  return false;
}
