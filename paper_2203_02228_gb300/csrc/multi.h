// multi.h -- host side of running many colonies through the same launches
// (the batch of faco_batch.h and the request server of faco_serve.h).
//
//   Group   colonies set up together: one device arena, laid out type by
//           type, holding their descriptors, lists, pheromone, tours and
//           set-up scratch; the whole set-up of Alg 2 is enqueued for all of
//           them with one launch per step and no host synchronisation.
//   AntSet  the per-ant buffers of a group for one ant count (second arena).
//   Runner  one iteration of Alg 2 for any list of colonies (of one or more
//           groups): descriptor tables, block maps, the redo list.
//   Tuner   per size class and ant count, which per-ant kernel is faster.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "faco.h"
#include "launch.h"

namespace faco {

constexpr int kMultiMaxN = 262144;  // shared-memory visited bits (ants, nearest-neighbour tour)
constexpr int kRedoBlocks = 38;     // blocks of the array kernel that serve the redo list

// Device-memory source for arenas (the batch: cudaMalloc; the server: its pool).
struct DevAlloc {
  virtual ~DevAlloc() {}
  virtual void* get(size_t bytes) = 0;  // nullptr when it does not fit
  virtual void put(void* p) = 0;
};

struct Group {
  int count = 0, kw = 16, max_n = 0;
  faco_params prm{};
  std::vector<int32_t> n, k, bl;
  std::vector<uint64_t> seed;
  std::vector<Colony> hC;       // descriptors as uploaded (grid: filled on the device)
  std::vector<ColonySetup> hS;
  std::vector<int64_t> node_off;  // prefix of n (packed tour output)
  char* base = nullptr;
  size_t bytes = 0, zero_bytes = 0;
  Colony* dC = nullptr;
  ColonySetup* dS = nullptr;
  int2* map256 = nullptr;
  int2* map128 = nullptr;
  int nmap256 = 0, nmap128 = 0;
  int64_t* d_node_off = nullptr;  // node_off on the device
};

struct AntSet {
  int m = 0;
  char* base = nullptr;
  size_t bytes = 0, zero_bytes = 0;
  std::vector<Ants> hA;         // with segment tables where cap > 0
  std::vector<int32_t> cap;
};

// Validates and fills the host side of a group (no device work).
int group_init(Group& g, const int32_t* ns, int count, int k, const faco_params& prm, const uint64_t* seeds);
// Arena size (base == nullptr) or pointers into base.
void group_layout(Group& g, char* base);
// Every coordinate in [0, 2^24), no NULL array.
int group_check_coords(const Group& g, const int32_t* const* coords);
// Coordinates from host memory (checked), then the set-up kernels.
int group_setup(Group& g, const int32_t* const* coords, cudaStream_t s);

// Segment-table capacity of colony i for the batch kernel's shared memory.
int ant_cap(int n, size_t smem_blk, int seg_mode);
void antset_layout(AntSet& a, const Group& g, int m, size_t smem_blk, int seg_mode, char* base);
int antset_zero(const AntSet& a, cudaStream_t s);

struct RunEntry {
  const Group* g;
  int i;                        // colony within g
  const AntSet* a;
  int variant;                  // kVariant*
};

// Per-ant kernel of a colony: a block of eight warps per ant on a segment
// table, or one warp per ant on explicit arrays with the kernel compiled for
// 2, 4 or 8 resident blocks per SM.
enum : int { kVarTable = 0, kVarArr2 = 1, kVarArr4 = 2, kVarArr8 = 3, kNVariants = 4 };
constexpr int kArrMinBlocks[kNVariants] = {0, 2, 4, 8};

struct Runner {
  int count = 0, kw = 16, nblk = 0, nmap256 = 0, redo_blocks = 0;
  int narr[kNVariants] = {0, 0, 0, 0};
  size_t smem_blk = 0, per_warp = 0;
  char* mem = nullptr;          // one cudaMalloc: tables, maps, redo list
  size_t mem_bytes = 0;
  Colony* dC = nullptr;
  Ants* dA = nullptr;
  int2* map_arr[kNVariants] = {nullptr, nullptr, nullptr, nullptr};
  int2 *map_blk = nullptr, *map256 = nullptr, *redo_list = nullptr;
  int32_t* redo_n = nullptr;
  // the per-ant launches of different kernels run side by side: forked from
  // and joined back into the caller's stream with events (graph branches
  // when captured)
  cudaStream_t side[kNVariants] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kNVariants] = {nullptr, nullptr, nullptr, nullptr};
  ~Runner();
  // Builds tables and maps for `entries` (enqueued on s).
  int build(const std::vector<RunEntry>& entries, size_t smem_blk, cudaStream_t s);
  // One iteration (per-ant kernels, then the colony update); parts: 1 ants, 2 update.
  int enqueue(cudaStream_t s, int parts = 3) const;
  int kernels_per_iteration() const;
};

// Size class of an instance for the tuner (factors of 4 in n).
int size_class(int n);
// Tuner objective: a batch's throughput (a size class's time scaled by the
// share of the GPU's resident ant slots it holds, the rest serving the
// other classes) or one request's latency (its time alone).
enum TuneGoal { kTuneBatch = 0, kTuneLatency = 1 };
// Cached choice for (size class, ants, roulette width, goal) on this
// device; -1 if none.
int tuner_get(int cls, int m, int kw, int goal = kTuneBatch);
void tuner_put(int cls, int m, int kw, int variant, int goal = kTuneBatch);
// Times every per-ant kernel on the colonies of each untuned size class of
// `entries` (per-ant buffers only are written) and records the best for
// the goal.
int tuner_run(const std::vector<RunEntry>& entries, size_t smem_blk, cudaStream_t s, int goal = kTuneBatch);
// Rows of (class, ants, roulette width, goal, chosen variant, the variants'
// timings in ms) for the current device, up to max_rows into out (5 +
// kNVariants doubles each); returns the number of rows recorded.
int tuner_report(double* out, int max_rows);

size_t batch_smem_blk(int kw);

// Range checks of faco_params shared by every constructor.
int check_faco_params(const faco_params& p);

}  // namespace faco
