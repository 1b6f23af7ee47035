// tiles.h - the 24 tile configurations shared by every stencil kernel.
//
// tile_id = 4 * shape + 2 * long_march + vec:
//   shape (threads bx x by): 32x4, 32x8, 64x4, 64x8, 128x2, 128x4
//   long_march: 0 -> zc = 16, 1 -> zc = 64   (planes per CTA in 3D;
//               2D kernels march zc / 4 rows per thread)
//   vec:        0 -> one element per thread in x, 1 -> a 16-byte vector
//               (2 doubles or 4 floats)
#pragma once

#define JACC_TILE_LIST(X)                                                                     \
  X(0, 32, 4, 0, 16) X(1, 32, 4, 1, 16) X(2, 32, 4, 0, 64) X(3, 32, 4, 1, 64)                \
  X(4, 32, 8, 0, 16) X(5, 32, 8, 1, 16) X(6, 32, 8, 0, 64) X(7, 32, 8, 1, 64)                \
  X(8, 64, 4, 0, 16) X(9, 64, 4, 1, 16) X(10, 64, 4, 0, 64) X(11, 64, 4, 1, 64)              \
  X(12, 64, 8, 0, 16) X(13, 64, 8, 1, 16) X(14, 64, 8, 0, 64) X(15, 64, 8, 1, 64)            \
  X(16, 128, 2, 0, 16) X(17, 128, 2, 1, 16) X(18, 128, 2, 0, 64) X(19, 128, 2, 1, 64)        \
  X(20, 128, 4, 0, 16) X(21, 128, 4, 1, 16) X(22, 128, 4, 0, 64) X(23, 128, 4, 1, 64)

#define JACC_NTILES 24
