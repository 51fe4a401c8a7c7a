// Multifrontal LU of the local Oseen systems (Algorithm 3 Step 3(2), eq. uclocalFully):
// nested-dissection symbolic analysis on the host, dense fronts factorised on the device.
//
// The unknowns of a local problem live on the half-grid of its box (P2 nodes; vertices at
// even coordinates).  A plane of vertices at an even coordinate separates the nodes on its
// two sides: no element holds nodes from both.  Recursive bisection of the box at such
// planes gives the elimination tree; every tree node owns the unknowns of its separator (a
// leaf owns its whole box) and eliminates them in one dense front.  Inside a front the
// velocities come before the pressures, so every pressure pivot follows eliminated
// velocities it is coupled to and the factorisation needs no pivoting (the static order
// the band LU also relies on).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace tpns {

constexpr int MF_NB = 32;      // pivot block (panel width) of the front factorisation
constexpr int MF_TILE = 128;   // rows / columns of one trailing-update tile
constexpr int MF_PACK_TILE = MF_TILE * MF_NB;   // elements of one packed operand tile
constexpr int MF_BIG_LIST = 1024;  // fronts per launch of the large-front path at most

struct MFFront {
  int m = 0, p = 0;              // front order, pivots (own unknowns)
  int level = 0;                 // height in the tree: leaves 0
  int parent = -1;
  int nchild = 0, child[2] = {-1, -1};
  std::vector<int32_t> rows;     // m unknowns: own (elimination order), then the update set
  std::vector<int32_t> relmap;   // update set (m - p entries) -> index in the parent's rows
  // originals: per column j, CSR entries (index into the system's values, row in front)
  std::vector<int32_t> col_ptr;  // m + 1
  std::vector<int32_t> orig_k, orig_i;
  std::vector<int32_t> col_child;   // m x 2: column of child c mapped onto column j, or -1
};

struct MFSymbolic {
  std::vector<MFFront> fronts;   // postorder (children before parents)
  std::vector<int32_t> order;    // elimination position -> unknown
  int nlevels = 0;
  double flops = 0;              // sum over fronts of sum_{k<p} (r + 2 r^2), r = m - 1 - k
  double factor_entries = 0;     // stored L and U entries: sum p^2 + 2 p (m - p)
};

// Nested dissection of one system.  coord: n x dim integer half-grid coordinates of the
// unknowns (vertices even); pressure[i] != 0 for pressure unknowns (eliminated after the
// velocities of their front); rowptr / colidx: a structurally symmetric CSR pattern.
// leaf_max: boxes with at most this many unknowns are not split further.
// Returns "" or an error message.
std::string mf_analyse(int n, int dim, const int32_t* coord, const int8_t* pressure, const int32_t* rowptr,
                       const int32_t* colidx, int leaf_max, MFSymbolic& out);

// Device descriptor of one front (offsets in elements of the front's precision T unless
// said otherwise).  The fronts of all systems are numbered in a topological order (every
// child precedes its parent), longest estimated remaining chain to the root first.
struct MFFrontDev {
  int64_t f_off;      // dense front, column-major, leading dimension ld
  int64_t dinv_off;   // per pivot block: L11^{-1} (32x32, row-major) then U11^{-1}
  int64_t upd_off;    // solve: update vector (m - p entries, T)
  int32_t m, p, ld, sys;
  int32_t nchild, child0, child1, parent;
  int32_t rows_off;   // the front's m unknowns start at rows_off
  int32_t relmap_off; // relmap of this front (m - p entries)
  int32_t colptr_off; // m + 1 column pointers into the originals
  int32_t pad;
};

// One system: its unknown vectors and CSR values.
struct MFSysDev {
  int32_t sid, n;     // system index (status / done words), unknowns
  int64_t x_off;      // unknown vectors of the system
  int64_t val_off;    // CSR values of the system
};

// Device arrays of the fronts of a set of systems, as the kernels read them.
struct MFLaunch {
  const MFSysDev* sys;
  int nsys;
  const MFFrontDev* fronts;
  int nfront;
  const int32_t* rows;      // per front: m unknowns (system numbering)
  const int32_t* relmap;
  const int64_t* colptr;
  const int32_t* orig_k;    // CSR value index within the system
  const int32_t* orig_ij;   // row | column << 16 in the front
  const double* vals;       // CSR values (all systems)
  int* status;              // per system: bit 0 bad pivot, bit 1 / 2 a bounded wait gave up
  int* sched;               // 8 ints: factor counter, finished CTAs, epoch; the same for the solves
  int* fflag;               // per front: epoch of its factorisation
  int* sflag;               // 2 per front: epochs of its forward and backward solve tasks
  int grid_cap;             // CTAs of a launch at most (0: as many as are resident at once)
};

}  // namespace tpns
