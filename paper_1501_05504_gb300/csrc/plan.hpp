// Host-side planning of the block-sparse contractions of the DMRG3S hot path.
//
// Every contraction is one of two three-stage pipelines that follow the
// optimal ordering (((L M) W) R) of Sec. V of arXiv:1501.05504:
//
//   left side  (H_eff application, expansion term for left-to-right sweeps,
//               left environment update):
//     stage 1  T1[bl, s]  = L[bl] . M[s]                       grouped GEMM
//     stage 2  T2[br, s'] = sum_{bl, s} W[s', s, bl, br] T1     combination
//     stage 3  HA[s']     = sum_{br} T2[br, s'] . R[br]^T       grouped GEMM
//           or L_i[br]    = sum_{s'} A[s']^T . T2[br, s']        grouped GEMM
//           or P          = alpha T2 written into the fused bond (stage 2 only)
//
//   right side (expansion term for right-to-left sweeps, right environment):
//     stage 1  U1[br, s]  = M[s] . R[br]^T                      grouped GEMM
//     stage 2  U2[bl, s'] = sum_{br, s} W[s', s, bl, br] U1     combination
//     stage 3  R_{i-1}[bl] = sum_{s'} B[s'] . U2[bl, s']^T       grouped GEMM
//           or P          = alpha U2 written into the fused bond
//
// A plan holds the task tables with element offsets relative to the base
// pointers of each stage (see the Kind comments), so that it can be reused
// for every call with the same block structure and MPO.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "kernels.hpp"
#include "layout.hpp"

namespace dmrg3s {

// Tensor-core form of a grouped GEMM stage (packed operands, 128 x 128 units).
struct TcStage {
  std::vector<TcSeg> segs;              // parallel to GemmStage::segs
  std::vector<TcUnit> units;            // grouped by CTA: CTA b runs units [cta_start[b], cta_start[b+1])
  std::vector<int32_t> cta_start;       // one entry per CTA of the persistent launch, plus one
  std::vector<PackBlock> packA, packB;  // empty for an operand packed by stage 2
  int64_t nA = 0, nB = 0;               // floats of one part (hi or lo) of each packed operand
  int32_t tilesA = 0, tilesB = 0;
};

struct GemmStage {
  Trans ta = Trans::N, tb = Trans::N;
  std::vector<GemmTask> tasks;
  std::vector<GemmSeg> segs;
  std::vector<GemmTile> tiles;      // 64 x 64 tiles (FP64 kernel)
  TcStage tc;
  double flops = 0.0;
  double bytes = 0.0;     // algorithmic: distinct operand blocks read once + output written once
  void add(int64_t offC, int ldc, int M, int N, const std::vector<GemmSeg>& s);
  void finalize_bytes(Trans ta, Trans tb);
};

struct CombStage {
  std::vector<CombTask> tasks;
  std::vector<CombTerm> terms;
  std::vector<CombChunk> chunks;
  double flops = 0.0;
  double bytes = 0.0;     // algorithmic: distinct input blocks read once + output written once
  void add(int64_t offOut, int ldo, int rows, int cols, const std::vector<CombTerm>& t);
};

enum class Kind {
  Heff,       // g1: A=L B=M C=ws1 | c2: ws1 -> ws2 | g3: A=ws2 B=R C=HA
  ExpandLR,   // g1 as Heff        | c2: ws1 -> P (scale alpha)
  EnvLR,      // g1, c2 as Heff    | g3: A=M B=ws2 C=L_out
  ExpandRL,   // g1: A=M B=R C=ws1 | c2: ws1 -> P (scale alpha)
  EnvRL       // g1, c2 as ExpandRL, c2 -> ws2 | g3: A=M B=ws2 C=R_out
};

struct Plan {
  Kind kind;
  GemmStage g1, g3;
  CombStage c2;
  bool has_g3 = false;
  int64_t ws1 = 0, ws2 = 0;     // doubles of the stage-1 / stage-2 intermediates
  int64_t nA1 = 0, nB1 = 0;     // elements of the stage-1 operand arrays
  int64_t nA3 = 0, nB3 = 0;     // elements of the stage-3 operand arrays (0 without stage 3)
  // Split-K form of stage 3 for the tensor-core kernel: one task per (output
  // block, K-segment) writing a double-float partial block, then a
  // deterministic sum.
  GemmStage g3s;                // partial products (C base = the partial buffer)
  CombStage c3r;                // sum of the partials into the output
  int64_t ws3 = 0;              // elements of the partial buffer
  // Tensor-core mode: stage 2 writes its output packed as the stage-3 operand
  // that is ws2 (A for Heff, B for EnvLR / EnvRL), one PackOut per c2 task.
  std::vector<PackOut> c2pack;
  int64_t nT2p = 0;             // floats of one part of the packed stage-2 output
  int32_t tilesT2 = 0;
  // Tensor-core H_eff (fused = true): stages 1 and 2 in one grouped GEMM g12
  // whose tasks are the T2 blocks and whose K-segments are the MPO terms,
  //   T2[br, s'] = sum_{(bl, s): W != 0} (W[s', s, bl, br] L[bl]) . M[s],
  // written packed (the c2pack placements) as the A operand of stage 3; T1 is
  // never formed.  g12's A operand is the coefficient-scaled L blocks.
  GemmStage g12;
  bool fused = false;
  double flops() const { return g1.flops + c2.flops + (has_g3 ? g3.flops : 0.0); }
};

// One plan of a merge and where its external operands sit in the merged
// operand arrays (element offsets).  oOut2 places the stage-2 output of the
// expansion kinds (P); for the kinds with stage 3 the stage-2 output is an
// intermediate and the stage-3 operand that reads it (A for Heff, B for the
// environments) is placed by the merge, so the corresponding field is unused.
struct PlanPart {
  const Plan* p = nullptr;
  int64_t oA1 = 0, oB1 = 0, oOut2 = 0, oA3 = 0, oB3 = 0, oC3 = 0;
  double c2scale = 1.0;     // folded into this part's MPO coefficients (the expansion's alpha)
};
// Plans of one kind side by side, as one plan: their task tables concatenated
// with every operand offset moved by its part's base (the parts'
// intermediates laid out back to back), then the split-K stage 3 and the
// tensor-core form built over the whole, so that one launch per stage
// serves every part.  n* are the sizes of the merged operand arrays.
dmrg3s_status merge_plans(Kind kind, const std::vector<PlanPart>& parts, int64_t nA1, int64_t nB1,
                          int64_t nOut2, int64_t nA3, int64_t nB3, int64_t nC3, Plan* out,
                          std::string* err);

// Number of CTAs of the persistent tensor-core launches (the SM count of the
// device; set when a context is created, 152 for a GB300).
void set_plan_ctas(int n);
int plan_ctas();

// Left-side plans.  `mps` is the site tensor M (or A); `le` its left
// environment (on mps.left, channels W.tl); `re` the right environment (on
// mps.right, channels W.tr) for Heff; `out_site` the layout of P for ExpandLR;
// `out_env` the layout of L_i for EnvLR.
dmrg3s_status plan_heff(const EnvLayout& le, const MpoLayout& W, const EnvLayout& re,
                        const SiteLayout& mps, Plan* plan, std::string* err);
dmrg3s_status plan_expand_lr(const EnvLayout& le, const MpoLayout& W, const SiteLayout& mps,
                             const SiteLayout& P, const FusedBond& fused, Plan* plan,
                             std::string* err);
dmrg3s_status plan_env_lr(const EnvLayout& le, const MpoLayout& W, const SiteLayout& mps,
                          const EnvLayout& out, Plan* plan, std::string* err);
dmrg3s_status plan_expand_rl(const EnvLayout& re, const MpoLayout& W, const SiteLayout& mps,
                             const SiteLayout& P, const FusedBond& fused, Plan* plan,
                             std::string* err);
dmrg3s_status plan_env_rl(const EnvLayout& re, const MpoLayout& W, const SiteLayout& mps,
                          const EnvLayout& out, Plan* plan, std::string* err);

// MPO-entry gradient of <M|H_eff|M> (the contraction of Sec. II with W_i
// taken out):
//   G[s', s, bl, br] = sum L[bl](al', al) M[s'](al', ar') M[s](al, ar) R[br](ar', ar)
// in three stages:
//   g1    T1[bl, s] = L[bl] . M[s]          (stage 1 of H_eff)    C = ws1
//   gy    Y[br, s'] = M[s'] . R[br]         (bra side through R)  C = wsy
//   dots  G[s', s, bl, br] = sum over the (al', ar) blocks of <T1[bl, s], Y[br, s']>
struct GradPlan {
  GemmStage g1, gy;
  std::vector<DotTask> tasks;     // one per entry of G, row-major [s'][s][bl][br]
  std::vector<DotSeg> segs;       // A = ws1, B = wsy
  int64_t ws1 = 0, wsy = 0, nG = 0;
  double dot_flops = 0.0;
  double flops() const { return g1.flops + gy.flops + dot_flops; }
};
dmrg3s_status plan_mpo_grad(const EnvLayout& le, const MpoLayout& W, const EnvLayout& re,
                            const SiteLayout& mps, GradPlan* plan, std::string* err);

// Structural compatibility checks shared by the entry points.
dmrg3s_status check_site_mpo(const SiteLayout& s, const MpoLayout& W, std::string* err);
dmrg3s_status check_env(const EnvLayout& e, const Bond& bond, int w,
                        const std::vector<Charge>& t, const char* what, std::string* err);

}  // namespace dmrg3s
