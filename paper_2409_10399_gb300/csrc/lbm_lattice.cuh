// Compile-time velocity sets of the three lattices the library instantiates.
//
// D1Q3 is given in App. A (Eq. (D1Q3lattice)); D2Q9 and D3Q19 are the
// standard sets the paper's any-dimension formulas are applied to.  Order:
// the rest velocity first, then the moving velocities in lexicographic order
// of (v_x, v_y, v_z) over {-1, 0, 1}^D (D3Q19: those with |v|^2 <= 2).  The
// set is symmetric under v -> -v and lexicographic order reverses under it,
// so opp(q) = Q - q for q > 0.  All accessors are constexpr so that, inside
// fully unrolled loops, every component and weight folds into the code.
#pragma once

namespace lbm {

constexpr double CS2 = 1.0 / 3.0;

template <int LAT> struct Lattice;

template <> struct Lattice<1> {
  static constexpr int D = 1, Q = 3;
  __host__ __device__ static constexpr int v(int q, int a) { return a != 0 ? 0 : (q == 1 ? -1 : (q == 2 ? 1 : 0)); }
  __host__ __device__ static constexpr double w(int q) { return q == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
  __host__ __device__ static constexpr int opp(int q) { return q == 0 ? 0 : Q - q; }
};

template <> struct Lattice<2> {
  static constexpr int D = 2, Q = 9;
  // q = 1..8 -> cell k of the 3x3 stencil without its centre (k = 4)
  __host__ __device__ static constexpr int cell(int q) { return q == 0 ? 4 : (q <= 4 ? q - 1 : q); }
  __host__ __device__ static constexpr int v(int q, int a) {
    return a == 0 ? cell(q) / 3 - 1 : (a == 1 ? cell(q) % 3 - 1 : 0);
  }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 4.0 / 9.0 : ((v(q, 0) != 0 && v(q, 1) != 0) ? 1.0 / 36.0 : 1.0 / 9.0);
  }
  __host__ __device__ static constexpr int opp(int q) { return q == 0 ? 0 : Q - q; }
};

template <> struct Lattice<3> {
  static constexpr int D = 3, Q = 19;
  // q = 1..18 -> cell k = 9(v_x+1) + 3(v_y+1) + (v_z+1) of the 3x3x3 stencil,
  // the 18 cells with 1 <= |v|^2 <= 2 in increasing order
  __host__ __device__ static constexpr int cell(int q) {
    return q == 0 ? 13
         : (q <= 5 ? (q == 1 ? 1 : (q == 2 ? 3 : (q == 3 ? 4 : (q == 4 ? 5 : 7))))
         : (q <= 13 ? (q == 6 ? 9 : (q == 7 ? 10 : (q == 8 ? 11 : (q == 9 ? 12 : (q == 10 ? 14 : (q == 11 ? 15 : (q == 12 ? 16 : 17)))))))
                    : (q == 14 ? 19 : (q == 15 ? 21 : (q == 16 ? 22 : (q == 17 ? 23 : 25))))));
  }
  __host__ __device__ static constexpr int v(int q, int a) {
    return a == 0 ? cell(q) / 9 - 1 : (a == 1 ? (cell(q) / 3) % 3 - 1 : cell(q) % 3 - 1);
  }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 1.0 / 3.0
                  : ((v(q, 0) * v(q, 0) + v(q, 1) * v(q, 1) + v(q, 2) * v(q, 2)) == 2 ? 1.0 / 36.0 : 1.0 / 18.0);
  }
  __host__ __device__ static constexpr int opp(int q) { return q == 0 ? 0 : Q - q; }
};

}  // namespace lbm
