// launch.h -- argument blocks shared by the host runtime and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace esbgk {

// Read-mostly view of a problem's device state.
struct View {
  Geo g;
  Model m;
  const double* eps;       // [nc] Knudsen number
  const uint8_t* flags;    // [nc] 1 = kinetic
  const int* klist;        // kinetic cells
  const int* blist;        // buffer cells (fluid, inside a kinetic stencil)
  const int* flist;        // other fluid cells
  const int* clist;        // cells that turned kinetic since the last step
  const int* counts;       // [4] nK, nB, nF, nC
  DevErr* err;
  // solid obstacles (null: none): per axis (x, y) and stencil offset (-2, -1,
  // +1, +2) the source cell of every cell's stencil value, [2][4][nc], and
  // whether it is a mirror image across a wall (specular reflection), [2][4][nc]
  const int* wsrc;
  const uint8_t* wrefl;
  const uint8_t* solid;  // [nc] 1 = solid cell (no state, never kinetic or fluid)
};

// One stage (or the final combination) of the IMEX step; see the stage
// kernel.  For kinetic cells:
//   L     = L(f_src)                              (none when f_src == null)
//   f*    = star_base + star_cL * L
//   f     = relax(f*, h = h_coef * nu)            (h_coef > 0), else f*
//   Q     = nu (G_hat - f)                        (h_coef > 0 or need_q)
//   acc_out[t] = acc_in[t] + acc_cL[t] L + acc_cQ[t] Q
//   f_out = f;  U_out = moments(f*) if kin_u_moments else U^n;
//   l1_out = ||f - M_hat[f]||_{L1_v} when set and there is no collision term
// For fluid cells: Phi[phi_store] = Phi(U_prev) (phi_store >= 0), then
//   U_out = U^n - sum_{j < nphi} phi_coef[j] Phi[j]; buffer cells also get
//   f_out = M_hat[U_out] (hoc) or M_hat[U^n] when `fill`.
struct StageArgs {
  const void* f_src;
  const void* star_base;
  double star_cL;
  double h_coef;
  int need_q;
  void* f_out;
  int nacc;
  const void* acc_in[3];
  void* acc_out[3];
  double acc_cL[3], acc_cQ[3];
  const double* Un;
  const double* U_prev;
  double* U_out;
  double* Phi;
  int phi_store;
  int nphi;
  double phi_coef[4];
  int hoc;
  int fill;
  int kin_u_moments;
  int iface;  // conservative interface: a buffer cell's Euler flux at a face with a kinetic neighbour is the
              // moments of the kinetic numerical flux there (computed from f_src)
  long long* ctr;
  double* l1_out;  // when set (final combination only): ||f - M_hat[f]||_L1 of the result per kinetic cell
  int* wq;         // work counter of the launch (zeroed by the step's prep): units past the first wave are
                   // claimed from it; null: static round-robin
  // float copies of the stage coefficients for the FP32 arithmetic
  float f_star_cL, f_h_coef, f_acc_cL[3], f_acc_cQ[3];
  // BF16 storage: stochastic rounding keyed by the step counter (advanced by
  // the step's prep kernel) and this launch's position in the step
  const unsigned* seed;
  unsigned sid;
};

// Start-of-step preparation: f := M_hat[U] in the cells of list1 and list2;
// copy_to := U (all cells) and flags_prev := flags when those are non-null.
struct PrepArgs {
  void* f;
  const double* U;
  int* wq_zero;  // work counters of the step's stage launches, zeroed here (wq_n of them)
  int wq_n;
  unsigned* seed;  // step counter of the stochastic rounding (may be null; advanced by a launch of its own)
  const int* list1;
  const int* count1;
  const int* list2;
  const int* count2;
  double* copy_to;
  uint8_t* flags_prev;
};

// Compile-time shapes of a kinetic stage launch.  The inner loops test none
// of these flags when they are fixed at compile time; kGeneric reads them all
// at run time and serves any other tableau.
enum StageMode : int {
  kGeneric = 0,
  kFirstRelax2 = 1,   // f* from f_src; relaxation; two accumulators started from f_src (ARS stage 2)
  kLoadedRelax1 = 2,  // f* from a loaded accumulator; relaxation; one loaded accumulator (ARS stage 3)
  kFinal = 3,         // no collision term; f* from a loaded accumulator; no accumulator (final combination)
  kFirstRelax0 = 4,   // f* from f_src; relaxation; no accumulator (stiffly accurate last stage)
  kNumModes = 5
};

// Per-cell code of a kinetic stage launch: the scalar form, or the vector
// form with groups of the widest vector (16 bytes of f, at most 4 nodes) or
// of 2 nodes, with one cell per warp or two (one per half-warp).  "Sx": one
// group of each velocity row straddles v_x = 0 (N_v/2 not a multiple of the
// group width); the other forms are compiled without that case.
enum StageVariant : int {
  kVarScalar = 0,
  kVarWide = 1,
  kVarWidePair = 2,
  kVarWideSx = 3,
  kVarWideSxPair = 4,
  kVarNarrowSx = 5,
  kVarNarrowSxPair = 6,
  kNumVariants = 7
};
__host__ __device__ inline bool variant_pairs(int v) {
  return v == kVarWidePair || v == kVarWideSxPair || v == kVarNarrowSxPair;
}

// Host-side choice of the specialisation for a launch.
inline int stage_mode(const StageArgs& A) {
  const bool relax = A.h_coef > 0.0;
  if (!A.f_src) return kGeneric;
  const bool bsrc = A.star_base == A.f_src;
  // (kFirstRelax2 rebuilds its accumulators from f* and f_src: it needs a transport coefficient)
  if (bsrc && relax && A.nacc == 2 && A.acc_in[0] == A.f_src && A.acc_in[1] == A.f_src && A.star_cL != 0.0)
    return kFirstRelax2;
  if (!bsrc && relax && A.nacc == 1 && A.acc_in[0] != A.f_src) return kLoadedRelax1;
  if (!bsrc && !relax && !A.need_q && A.nacc == 0) return kFinal;
  if (bsrc && relax && A.nacc == 0) return kFirstRelax0;
  return kGeneric;
}

// ---------------------------------------------------------------------------
// Batched form: many independent cases advanced by one launch per kernel.
// Every per-case descriptor lives in device memory; a global work unit u
// belongs to the case c with off[c] <= u < off[c+1].

// Shared memory the batched kernels reserve for their per-warp descriptor
// copies; the dynamic f-sized arrays get the rest of the opt-in limit.
constexpr int kBatchStaticSmem = 8 * 1024;
// Vector-form stage kernels run two kinetic cells per warp (16 lanes each)
// when the velocity grid has at most this many nodes.
constexpr int kPairMaxNodes = 512;

// One case of a batched stage launch (vec: the vector node-group form applies).
struct CaseStage {
  View V;
  StageArgs A;
  int variant;  // StageVariant of the case (the same for every launch of the step)
  int pad;
};

// One case of a batched start-of-step launch.
struct CasePrep {
  View V;
  PrepArgs P;
};

// One case of the batched regime update.
struct CaseRegime {
  View V;
  const void* f;          // f^n
  double* Un;
  double* L1;
  double* lamA;
  uint8_t* flags;
  uint8_t* flags_prev;
  uint8_t* cat;
  int* klist;
  int* blist;
  int* flist;
  int* clist;
  int* counts;
  int* l1_fresh;          // device flag: L1 already holds the deviation of f^n
  int plain;              // plain switch (else the regime map is kept)
  int l1_next;            // the final combination of this step computes L1
  int prep_copy;          // the start-of-step launch copies U^n and flags (units of 32 cells)
  int conv;               // the start-of-step launch fills converted cells
  int variant;            // StageVariant of the case's stage launches
  int learned;            // learned switch: 1, 2 when the previous prediction is judged; else 0
};

// Device tables of a batch.
struct BatchTabs {
  const CaseRegime* reg;  // [n]
  const int* cell_off;    // [n+1] prefix of cells
  int* off_stage;         // [kNumVariants][n+1] prefix of stage units (cases of other variants: none)
  int* off_prep;          // [n+1] prefix of start-of-step units
  int* off_l1;            // [n+1] prefix of L1 units
  int n;
  int total_cells;
  int fp32;  // the criterion's arithmetic in float32 (FP32 and BF16 storage)
};

// Per-storage-type launchers (one table per precision).
struct Launchers {
  size_t elem;
  cudaError_t (*setup)(const Geo&);
  int (*blocks_per_sm)(const Geo&);
  void (*stage)(const StageArgs&, const View&, int grid, cudaStream_t);
  void (*prep)(const PrepArgs&, const View&, int grid, cudaStream_t);
  void (*l1)(const void* f, const double* U, double* L1, const View&, int grid, cudaStream_t);
  void (*relax_cells)(const void* fs, const double* h, int n, const Geo&, double beta, void* fo, void* go,
                      int grid, cudaStream_t);
  void (*moments)(const void* f, double* U, const View&, int grid, cudaStream_t);
  // batched form; threads per CTA (multiple of 32, <= 128) and grid chosen by the caller;
  // comp: some case asks for compensated moment sums
  void (*batch_stage)(const CaseStage* cases, const int* off, int n, int mode, int var, bool comp, int max_nvv,
                      int threads, int grid, cudaStream_t);
  void (*batch_prep)(const CasePrep* cases, const int* off, int n, int grid, cudaStream_t);
  void (*batch_l1)(const CaseRegime* cases, const int* off, int n, int max_nvv, int grid, cudaStream_t);
  int (*batch_stage_occupancy)(int mode, int var, bool comp, int max_nvv, int threads);
  int (*variant)(const StageArgs& A, const Geo& g);
  int wide_nodes;  // nodes per group of the kVarWide variants
  // tiled stage kernel for problems whose every cell is kinetic (regime frozen)
  int (*tile_ok)(const StageArgs& A, const Geo& g);
  void (*stage_tile)(const StageArgs&, const View&, int grid, cudaStream_t);
};

extern const Launchers kLaunchF64;
extern const Launchers kLaunchF32;
extern const Launchers kLaunchBF16;

// Precision-independent kernels (kernels_common.cu).
void launch_init_state(const double* prim /*[5][nc] rho ux uy T eps*/, const uint8_t* kin_in, double* Un,
                       double* eps, uint8_t* flags, uint8_t* flags_prev, int nc, cudaStream_t s);
// fp32: the criterion's arithmetic in float32 (FP32 and BF16 storage), else float64.
void launch_flags(const View& V, const double* Un, const double* L1in, double* L1out, double* lamA,
                  uint8_t* flags_out, bool fp32, cudaStream_t s);
void launch_categorize(const View& V, const uint8_t* flags, const uint8_t* flags_prev, uint8_t* cat,
                       cudaStream_t s);
void launch_compact(const uint8_t* cat, int nc, int* klist, int* blist, int* flist, int* clist, int* counts,
                    cudaStream_t s);
// categories (into cat) and lists in ascending cell order, fully parallel;
// block_counts holds 4 * categorize_blocks(nc) ints
void launch_categorize_compact(const View& V, const uint8_t* flags, const uint8_t* flags_prev, uint8_t* cat,
                               int* block_counts, int* klist, int* blist, int* flist, int* clist, int* counts,
                               cudaStream_t s);
int categorize_blocks(int nc);
// One CTA waiting on a barrier with the bounded wait (limit polls); arrive = 0
// withholds the arrival.  *err_out: 0, or kErrTimeout when the wait ran out.
cudaError_t launch_wait_probe(int arrive, unsigned limit, int* err_out, cudaStream_t s);
void launch_prim(const double* Un, double* out /*[4][nc]*/, int nc, cudaStream_t s);
// flags and flags_prev := 0 in solid cells
void launch_clear_solid(uint8_t* flags, uint8_t* flags_prev, const uint8_t* solid, int nc, cudaStream_t s);
// advance the step counter of the stochastic rounding (one thread)
void launch_seed_advance(unsigned* seed, cudaStream_t s);
// solid (may be null): cells left out of the totals
void launch_totals(const double* Un, const uint8_t* solid, int nc, double* partial /*[grid][4]*/, double* out,
                   double dxdy, int grid,
                   cudaStream_t s);
// batched regime update: offsets of the L1 units, flags, categories,
// compaction (one CTA per case), offsets of the stage and start-of-step units
void launch_batch_l1_offsets(const BatchTabs& T, cudaStream_t s);
void launch_batch_flags(const BatchTabs& T, cudaStream_t s);
void launch_batch_categorize(const BatchTabs& T, cudaStream_t s);
void launch_batch_compact(const BatchTabs& T, cudaStream_t s);
void launch_batch_offsets(const BatchTabs& T, cudaStream_t s);
// advance every case's stochastic-rounding counter (cases with a counter)
void launch_batch_seed_advance(const CasePrep* cases, int n, cudaStream_t s);

}  // namespace esbgk
