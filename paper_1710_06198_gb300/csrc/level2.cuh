// Index helpers of the third level (internal).  Level-1 sites are numbered lexicographically on the
// level-1 lattice NB (x fastest); level-2 aggregates are A-shaped blocks of level-1 sites,
// numbered lexicographically on the level-2 lattice NA.
#pragma once

namespace tmg {

struct L2Geom {
  int NB[4];     // level-1 lattice
  int A[4];      // level-2 aggregate (in level-1 sites)
  int NA[4];     // level-2 lattice
  int nc1, nd1, nv1, nc2, nv2, avol;
};

__device__ __forceinline__ void l1_coords(const L2Geom& q, int a1, int c[4]) {
  c[0] = a1 % q.NB[0]; a1 /= q.NB[0];
  c[1] = a1 % q.NB[1]; a1 /= q.NB[1];
  c[2] = a1 % q.NB[2]; c[3] = a1 / q.NB[2];
}

__device__ __forceinline__ int l2_agg_of(const L2Geom& q, const int c[4]) {
  return (c[0] / q.A[0]) + q.NA[0] * ((c[1] / q.A[1]) + q.NA[1] * ((c[2] / q.A[2]) + q.NA[2] * (c[3] / q.A[3])));
}

// level-1 site of local index t (x fastest) inside level-2 aggregate a2
__device__ __forceinline__ int l2_member(const L2Geom& q, int a2, int t) {
  int b[4], l[4];
  b[0] = a2 % q.NA[0]; a2 /= q.NA[0];
  b[1] = a2 % q.NA[1]; a2 /= q.NA[1];
  b[2] = a2 % q.NA[2]; b[3] = a2 / q.NA[2];
  l[0] = t % q.A[0]; t /= q.A[0];
  l[1] = t % q.A[1]; t /= q.A[1];
  l[2] = t % q.A[2]; l[3] = t / q.A[2];
  const int c0 = b[0] * q.A[0] + l[0], c1 = b[1] * q.A[1] + l[1], c2 = b[2] * q.A[2] + l[2], c3 = b[3] * q.A[3] + l[3];
  return c0 + q.NB[0] * (c1 + q.NB[1] * (c2 + q.NB[2] * c3));
}

struct Ctx;
// geometry of the built hierarchy (cl, cl2 and the fine geometry's level-1 lattice)
L2Geom l2geom(const Ctx& c);

}  // namespace tmg
