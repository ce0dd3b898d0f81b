// bfs_kernels_lean.cu -- the single-source persistent traversal kernel built
// without the paths it only takes when a run asks for them (direction
// optimisation and frontier bitmaps, the shared-memory hot bitmap,
// warp-aggregated claims, bulk L2 prefetch), into namespace bfs::lean.  The
// host launches it for every traversal that uses none of them.
#define BFS_LEAN_PATHS 1
#include "bfs_kernels.cu"
