// Compile-time velocity sets of the three lattices the library instantiates.
//
// D1Q3 is given in App. A (Eq. (D1Q3lattice)); D2Q9 and D3Q19 are the
// standard sets the paper's any-dimension formulas are applied to.  Opposite
// directions are stored next to each other (q, q+1 for odd q), so
// opp(q) = q + 1 for odd q and q - 1 for even q > 0.  All accessors are
// constexpr so that, inside fully unrolled loops, every velocity component
// and weight folds into the instruction stream.
#pragma once

namespace lbm {

constexpr double CS2 = 1.0 / 3.0;

__host__ __device__ constexpr int opp_of(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }

template <int LAT> struct Lattice;

template <> struct Lattice<1> {
  static constexpr int D = 1, Q = 3;
  __host__ __device__ static constexpr int v(int q, int a) {
    return a != 0 ? 0 : (q == 1 ? 1 : (q == 2 ? -1 : 0));
  }
  __host__ __device__ static constexpr double w(int q) { return q == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
};

template <> struct Lattice<2> {
  static constexpr int D = 2, Q = 9;
  // 0 rest; 1,2 = +-x; 3,4 = +-y; 5,6 = +-(1,1); 7,8 = +-(1,-1)
  __host__ __device__ static constexpr int v(int q, int a) {
    return a == 0 ? ((q == 1 || q == 5 || q == 7) ? 1 : ((q == 2 || q == 6 || q == 8) ? -1 : 0))
         : a == 1 ? ((q == 3 || q == 5 || q == 8) ? 1 : ((q == 4 || q == 6 || q == 7) ? -1 : 0))
                  : 0;
  }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

template <> struct Lattice<3> {
  static constexpr int D = 3, Q = 19;
  // 0 rest; 1..6 = +-x, +-y, +-z; 7..18 = +-(1,1,0), +-(1,-1,0), +-(1,0,1),
  // +-(1,0,-1), +-(0,1,1), +-(0,1,-1)
  __host__ __device__ static constexpr int v(int q, int a) {
    return a == 0 ? ((q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
                   : ((q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0))
         : a == 1 ? ((q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
                   : ((q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0))
                  : ((q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
                   : ((q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0));
  }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

}  // namespace lbm
