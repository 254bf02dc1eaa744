// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rad.h"

namespace rad {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxBinsStep = 812;        // rad_step: one CTA of <= 512 threads holds all bins of a cell
                                         // (812 = geodesic level 9)
constexpr int kMaxSlots = 6;             // neighbours of a geodesic cell
constexpr int kMaxBehind = 4;            // sides whose line reconstruction reads a lat/long cell as
                                         // the cell behind (one per line direction)

// error bits of the sticky device word (bit k <-> status -k)
constexpr int kErrNoConv = 1 << 4;       // RAD_ENOCONV = -4
constexpr int kErrNonFinite = 1 << 5;    // RAD_ENONFINITE = -5
constexpr int kErrState = 1 << 6;        // RAD_ESTATE = -6: tables inconsistent with the kernel's assumptions

// Host description of the geodesic grid (Sec. 2.6); built by angles.cpp.
struct AngleGrid {
  int level = 0, n_ang = 0, n_ap = 0, n_edge = 0;
  bool sign_pairs = false;        // bins 2t, 2t + 1 have no direction component of opposite sign
  std::vector<double> dir;        // [n_ang][3]
  std::vector<double> dOmega;     // [n_ang]
  std::vector<int> nbr;           // [n_ang][6], -1 padded
  std::vector<int> edge_pq;       // [n_edge][2], p < q
  std::vector<double> edge_mid;   // [n_edge][3]
  std::vector<double> edge_nrm;   // [n_edge][3], from p to q
  std::vector<double> edge_len;   // [n_edge]
  std::vector<int> slot_edge;     // [n_ang][6] edge id of each neighbour slot (-1 pad)
  std::vector<int> perm;          // [n_ang] bin of the pi-rotation about 2hat
  std::vector<int> edge_line;     // [n_edge][2] cell behind p, cell beyond q on the line through the
                                  // side (latitude-longitude grids; empty for the geodesic grid)
  std::vector<int> mapr_nb;       // [n_ang][6] neighbours in cyclic order (-1 pad; geodesic grids)
  std::vector<double> mapr_minv;  // [n_ang][6][4] inverse of [x_a; x_b] of plane a (gnomonic x)
  std::vector<double> mapr_xo;    // [n_ang][6][2] gnomonic x of slot s's side midpoint, own plane
  std::vector<double> mapr_xn;    // [n_ang][6][2] the same midpoint in the neighbour's plane
  std::vector<int> line_behind;   // [n_ang][kMaxBehind] 2 e + s for every side e whose line
                                  // reconstruction from its cell s (0: p, 1: q) takes this bin as
                                  // the cell behind (-1 pad; latitude-longitude grids only)
};

bool build_geodesic(int level, AngleGrid &g, std::string &err);
bool build_latlong(int n_zeta, int n_psi, AngleGrid &g, std::string &err);

// Per-cell geometry of one (i, j) column (the metrics are x3-independent).
struct ColGeo {
  double n0up;      // n^0 = e^0_0hat (the same for every bin)
  double invdV;     // 1 / Delta V
  double dV;
  double M[4][4];   // M[mu][A] = g_{mu nu} e^nu_A, so n_mu = M[mu][A] n^A
  double e[4][4];   // e[mu][A] = e^mu_A
  double K[3][10];  // omega^ihat_{AB} n^A n^B = sum_p K[i-1][p] (n n)_p, p over
                    // (00,01,02,03,11,12,13,22,23,33), off-diagonals doubled
  double K0[10];    // the same for omega^0hat_{AB} n^A n^B (the frequency symbol n^nu = -nu K0 . (n n))
};

// Per-face geometry for the flux prefactor Delta A n^d n_0.
struct FaceGeo {
  double ea[4];     // e^d_A: row of the tetrad for the face's coordinate
  double m0[4];     // M[0][A] at the face (n_0 = m0 . n)
  double dA;        // exact face area (0 on a polar axis)
  double pad[3];
};

// Single-precision copies used by the FP32 kernels (same layout).
struct ColGeoF {
  float n0up, invdV, dV, pad;
  float M[4][4];
  float e[4][4];
  float K[3][10];
  float pad2[2];
  float K0[10];
  float pad3[2];
};
struct FaceGeoF {
  float ea[4];
  float m0[4];
  float dA, pad[3];
};

// Device copies of the angle tables.
struct DevAngles {
  double *dir = nullptr;       // [n_ap][3] (zeros in padding)
  double *dOmega = nullptr;    // [n_ap]
  int *slot_nbr = nullptr;     // [n_ap][6]
  int *slot_edge = nullptr;    // [n_ap][6]
  int *perm = nullptr;         // [n_ap]
  double *edge_geo = nullptr;  // [n_edge][8]: mid xyz, nrm xyz, len, p-index
  int *edge_pq = nullptr;      // [n_edge][2]
  int *edge_line = nullptr;    // [n_edge][2] (latitude-longitude grids only)
  int *line_behind = nullptr;  // [n_ap][kMaxBehind] (latitude-longitude grids only)
  int *mapr_nb = nullptr;      // [n_ap][6] (geodesic grids only)
  double *mapr_minv = nullptr; // [n_ap][6][4]
  double *mapr_xo = nullptr;   // [n_ap][6][2]
  double *mapr_xn = nullptr;   // [n_ap][6][2]
};

struct DevGeom {
  int ndim = 0, n[3] = {0, 0, 0};
  int bc_lo[3], bc_hi[3];
  int kind = 0;
  double spin = 0.0;
  std::vector<double> xf[3];
  ColGeo *cols = nullptr;      // [n2][n1]
  FaceGeo *f1 = nullptr;       // [n2][n1+1]
  FaceGeo *f2 = nullptr;       // [n2+1][n1]
  FaceGeo *f3 = nullptr;       // [n2][n1]
  ColGeoF *colsF = nullptr;    // float copies of the above
  FaceGeoF *f1F = nullptr, *f2F = nullptr, *f3F = nullptr;
  double *xf_dev = nullptr;    // packed face coordinates
};

}  // namespace rad

struct rad_ctx {
  cudaStream_t stream = nullptr;
  std::string last_error;
  rad::AngleGrid ang;
  rad::DevAngles dang;
  rad::DevGeom geom;
  bool have_angles = false, have_metric = false;
  int *err_word = nullptr;      // sticky device error bits
  // rad_step scratch: stage-1 intensity and temperature
  void *scratch_I = nullptr;
  size_t scratch_I_bytes = 0;
  double *scratch_T = nullptr;
  size_t scratch_T_count = 0;
  int stage1_prec = -1;         // precision of the last rad_step_stage stage 1 (its result is in scratch_I)
  // multigroup transport (rad_set_groups): 0 = gray; else the group count,
  // the n_groups + 1 frequency edges and the per-group frequency divergence
  int n_groups = 0;
  std::vector<double> nu_edges;
  double *nu_edges_dev = nullptr;
  void *freq_buf = nullptr;
  size_t freq_bytes = 0;
  // rad_step_adjoint scratch
  void *adj_buf = nullptr;
  size_t adj_bytes = 0;
  // split-bf16 moment weights (W^T hi / lo in the tensor-core operand layout)
  void *wt_dev = nullptr;
  int wt_kp = 0, wt_level = 0;
  // per-row partials of the outgoing-flux loss
  double *loss_buf = nullptr;
  int loss_rows = 0;
  // rad_step_host: kHostSlots device slots, the upload, read-back and moment
  // streams and the per-slot events
  static constexpr int kHostSlots = 3;
  void *host_slot_buf = nullptr;
  size_t host_slot_bytes = 0;
  cudaStream_t copy_stream = nullptr, back_stream = nullptr, mom_stream = nullptr;
  cudaEvent_t ev_h2d[kHostSlots] = {}, ev_step[kHostSlots] = {}, ev_done[kHostSlots] = {}, ev_back[kHostSlots] = {};
};

namespace rad {

// capi.cu: the checks shared by every RK2 step entry point (sets ctx->last_error)
// (staged: rad_step_stage, which takes blocks with faces shared with other blocks)
int check_step_args(rad_ctx *ctx, const void *I, const rad_gas *gas, double dt, const rad_opts *o,
                    bool staged = false);

// geom.cu
int compute_geometry(rad_ctx *ctx, std::string &err);
void free_geometry(DevGeom &g);

// step.cu
struct StageArgs;
int launch_step(rad_ctx *ctx, void *I, const rad_gas *gas, double dt, const rad_opts *opts,
                double *gas_src, void *scratch_I, double *scratch_T, std::string &err);
// one RK2 stage (1: I -> scratch, 2: scratch + I -> I); halo: the ghost rows of
// faces shared with other blocks (6 pointers, face (d, side) at 2 d + side), or null
int launch_stage_s(rad_ctx *ctx, int stage, void *I, const rad_gas *gas, double dt, const rad_opts *opts,
                   double *gas_src, void *scratch_I, double *scratch_T, const void *const *halo,
                   std::string &err);
// multigroup: the frequency divergence F_{g+1} - F_g of every group of I into D (frequency.cu)
int launch_freq_div(rad_ctx *ctx, const void *I, void *D, int precision, std::string &err);
// one RK2 step of every group (step.cu): frequency divergence, then the stage kernel per group
int launch_step_groups(rad_ctx *ctx, void *I, const rad_gas *gas, double dt, const rad_opts *opts,
                       double *gas_src, void *scratch_I, double *scratch_T, void *D, std::string &err);
// rad_gas_update (gas.cu)
int launch_gas_update(rad_ctx *ctx, double *rho, double *u, double *T, const double *src, int nsrc, double gamma,
                      std::string &err);
// rad_halo_pack: the kHaloLayers layers of I next to face (dim, side) into buf
int launch_halo_pack(rad_ctx *ctx, const void *I, int precision, int dim, int side, void *buf, std::string &err);
constexpr int kHaloLayers = 3;   // the widest stencil (PPM) reaches three cells
int launch_cfl(rad_ctx *ctx, double cfl, double *dt_out, std::string &err);
cudaError_t launch_wait_selftest(rad_ctx *ctx, double seconds);

// moments.cu
int launch_moments(rad_ctx *ctx, const void *I, int precision, int frame, int method,
                   const rad_gas *gas, void *R, cudaStream_t st, std::string &err);

// adjoint.cu
int launch_adjoint(rad_ctx *ctx, const void *I_n, const rad_gas *gas, double dt,
                   const rad_opts *opts, const void *lam_np1, void *lam_n, const double *lamT_np1,
                   double *lamT_n, double *g_aa, double *g_as, double *g_eta, std::string &err);
int launch_loss(rad_ctx *ctx, const void *I, int precision, double *L, void *dL, std::string &err);

}  // namespace rad
