/*
 * rv.h -- C ABI of librv, the GB300 (sm_103a) tree-gravity library.
 *
 * librv computes the data-parallel part of a regularised tree code's force
 * step (Karl et al., "introducing the regularized tree code rVINE"):
 *   - softened Barnes-Hut tree forces on the field stars (Sect. 2: forces of
 *     most particles from the tree with Plummer softening; Sect. 1: multipole
 *     expansion of a distant group about its centre of mass; Sect. 3: Plummer
 *     softening, G = 1) built from Morton keys, a radix sort and an octree
 *     with monopole and quadrupole moments, walked under an opening-angle
 *     test;
 *   - the unsoftened FP64 couplings between a regularised chain and its
 *     perturbers (Sect. 2, Eq. 3 and the text around it);
 *   - a kick-drift-kick step and FP64 energy/momentum totals.
 * The chain's own regularised integrator is not part of this library.
 *
 * Conventions (every entry point):
 *   - Pointers marked "device" are CUDA device addresses owned by the caller;
 *     librv never frees them. "host" pointers are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy stream). All
 *     device work is enqueued asynchronously on it; a call returns once the
 *     work is enqueued, except where a function says it synchronises.
 *   - Arrays of stars are in the caller's order; internal sorting never
 *     leaks out. Star data are FP32; chain data are FP64.
 *   - Errors are returned as rv_status and never abort or trap. Errors found
 *     by a kernel (a full walk stack, a tree larger than the workspace) are
 *     latched in device memory and reported by rv_sync_status().
 *   - Not thread safe per context; distinct contexts are independent.
 */
#ifndef RV_H
#define RV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RV_OK = 0,
    RV_E_INVAL = 1,     /* bad argument (null pointer, size out of range, bad config) */
    RV_E_CUDA = 2,      /* a CUDA runtime call failed; rv_last_error() has the text */
    RV_E_WORKSPACE = 3, /* workspace missing, too small, or the tree outgrew it */
    RV_E_STACK = 4,     /* a walk's traversal stack filled up (results invalid) */
    RV_E_TIMEOUT = 5,   /* a bounded device wait gave up */
    RV_E_NOTBUILT = 6,  /* forces asked before rv_build_tree */
    RV_E_TOO_LARGE = 7  /* input larger than a fixed-size internal buffer allows */
} rv_status;

typedef struct rv_ctx rv_ctx; /* opaque; owned by librv */

/* Tree parameters.
 *   theta      opening angle: a cell of side s is used as a multipole for a
 *              walk group when s < theta * d, d the distance between the
 *              group's box and the cell's box (0 <= theta < 2).
 *   eps_star   Plummer softening length of the stars (>= 0).
 *   n_leaf     a cell with more than n_leaf stars is split (1..64).
 *   group      stars per walk group, at most 64 (two per warp lane): runs of `group` consecutive
 *              stars in key order, each walked with the tightest integer-grid
 *              box of its stars as the group's box.
 *   quadrupole 1: monopole + traceless quadrupole; 0: monopole only.
 *   tile       interaction-list tile, a multiple of 32 in [32, 256].
 *   mac        opening criterion of rv_system_forces / rv_kdk_step(_graph):
 *              0 = opening angle theta; 1 = the relative criterion of
 *              rv_tree_forces_rel with tolerance `alpha`, the system's current
 *              accelerations (the previous pass's) as references; groups
 *              without a reference yet (|a| = 0) and the chain's
 *              centre-of-mass particles use theta.
 *   alpha      tolerance of the relative criterion (>= 0).
 *   softening  0 = Plummer (Sect. 3); 1 = spline (the "spline" option of
 *              Sect. 2): the cubic-spline field of support h = 2.8 eps_star
 *              (phi(0) = -m/eps_star as for Plummer), Newton beyond h; cells
 *              closer than h act as spline monopoles. */
typedef struct {
    float theta;
    float eps_star;
    int32_t n_leaf;
    int32_t group;
    int32_t quadrupole;
    int32_t tile;
    int32_t mac;
    float alpha;
    int32_t softening;
} rv_config;

/* Fills *cfg with the defaults: theta 0.5, eps 0.01, n_leaf 16, group 32,
 * quadrupole 1, tile 64, mac 0, alpha 1e-3, softening 0. */
void rv_default_config(rv_config *cfg);

/* Bytes of device workspace a context needs for up to n_max stars (0 if the
 * config is invalid). */
size_t rv_workspace_size(int64_t n_max, const rv_config *cfg);

/* Creates a context for up to n_max stars on the current CUDA device.
 * Allocates only small host state; device memory comes from
 * rv_set_workspace. Returns RV_E_INVAL for a bad config or n_max < 0. */
rv_status rv_create(rv_ctx **out, int64_t n_max, const rv_config *cfg);
void rv_destroy(rv_ctx *ctx);

/* Hands librv `bytes` of caller-owned device memory (256-byte aligned), at
 * least rv_workspace_size(). Must stay valid until rv_destroy or the next
 * rv_set_workspace. RV_E_WORKSPACE if too small or misaligned. */
rv_status rv_set_workspace(rv_ctx *ctx, void *dev, size_t bytes);

/* Builds the octree of n stars (device FP32 arrays x, y, z, m; n <= n_max).
 * Steps: bounding cube; 63-bit Morton keys q_a = min(floor((x_a - min_a)
 * 2^21 / L), 2^21 - 1) interleaved x, y, z from bit 0; stable radix sort;
 * gather of (x, y, z, m) in key order; cells = key prefixes split while they
 * hold more than n_leaf stars (down to level 21), breadth-first; per cell the
 * mass, centre of mass and traceless quadrupole about it (Sect. 1); walk
 * groups (runs of `group` stars and their boxes). Inputs are read during the call's stream work only. */
rv_status rv_build_tree(rv_ctx *ctx, int64_t n, const float *x, const float *y, const float *z,
                        const float *m, void *stream);

/* rv_build_tree for n_members independent members stored one after another
 * (host offsets[n_members + 1], offsets[0] = 0, non-decreasing,
 * offsets[n_members] = n <= n_max; 1 <= n_members <= 512). Every member gets
 * its own bounding cube, keys and tree, exactly as if built alone; they
 * share the launches. */
rv_status rv_build_tree_members(rv_ctx *ctx, int32_t n_members, const int64_t *offsets, const float *x,
                                const float *y, const float *z, const float *m, void *stream);

/* Tree forces on all stars of the last build (G = 1, Sect. 3):
 *   a_i = sum_j m_j r_ij / (r_ij^2 + eps^2)^{3/2},  phi_i = -sum_j m_j (r^2+eps^2)^{-1/2}
 * over the other stars, with distant cells replaced by their multipoles
 * under the opening test at `theta`, evaluated in FP32 with positions taken
 * relative to the target and compensated (Neumaier) accumulation per tile.
 * Outputs ax, ay, az, pot (device FP32 [n], caller order) are overwritten.
 *
 * n_extra (0..8) particles outside the tree -- a chain's centre-of-mass
 * particle (Sect. 2) -- are given as device FP32 xyzm[4 n_extra] and
 * eps[n_extra] (0 = unsoftened; pair softening max(eps_i, eps_j), 0 if either
 * is 0). They act on every star directly and feel the tree through their own
 * walk; their acceleration and potential go to device extra_out[4 n_extra]
 * (ax, ay, az, pot). extra pointers may be NULL when n_extra = 0. */
rv_status rv_tree_forces(rv_ctx *ctx, float theta, float eps_star, int32_t n_extra,
                         const float *extra_xyzm, const float *extra_eps, float *ax, float *ay,
                         float *az, float *pot, float *extra_out, void *stream);

/* Tree forces on all stars of the last build (members included) under the
 * relative opening criterion the paper's runs use (Sect. 3: a "Gadget"
 * criterion with an error tolerance; read as the Gadget-2 relative
 * criterion). A cell of mass M and side s is used as a multipole for a walk
 * group when
 *   M s^2 <= alpha |a| d^4   and the group's box lies outside the cell's box
 *                            grown by s/10 on every side,
 * d the box-box distance and |a| the smallest reference magnitude among the
 * group's stars: ref_ax, ref_ay, ref_az (device FP32 [n], caller order) hold
 * reference accelerations, normally the previous step's, and |a| =
 * sqrt((x x + y y) + z z). Every test runs in FP32 with one rounding per
 * operation: K = (alpha |a|min) (u u), u the grid unit, accept iff
 * M s^2 <= (K d^2) d^2 with d^2 in grid units. alpha = 0 gives the direct
 * sum. A group whose smallest reference magnitude is 0 (no force pass yet)
 * uses the opening angle of the context's configuration (theta).
 * Outputs as rv_tree_forces (no extra particles); the reference arrays
 * may be the output arrays themselves (each group reads its own stars'
 * references before it writes their forces). */
rv_status rv_tree_forces_rel(rv_ctx *ctx, float alpha, float eps_star, const float *ref_ax, const float *ref_ay,
                             const float *ref_az, float *ax, float *ay, float *az, float *pot, void *stream);

/* rv_tree_forces after rv_build_tree_members: each star feels only its own
 * member's tree and the extra particles of its member; extra k belongs to
 * member extra_member[k] (device int32 [n_extra]; NULL = member 0) and walks
 * that member's tree. */
rv_status rv_tree_forces_members(rv_ctx *ctx, float theta, float eps_star, int32_t n_extra,
                                 const float *extra_xyzm, const float *extra_eps, const int32_t *extra_member,
                                 float *ax, float *ay, float *az, float *pot, float *extra_out, void *stream);

/* Unsoftened FP64 chain/perturber coupling (Sect. 2, Eq. 3). Chain members k
 * (n_ch <= 250; device chain_m[n_ch], chain_x[3 n_ch]) with centre of mass
 * c and mass M; perturbers p (n_pert <= 5000; device FP64 pert_m[n_pert],
 * pert_x[3 n_pert]). Device FP64 outputs:
 *   a_pert[3p..], pot_pert[p]:  sum_k m_k f(x_k - x_p) - M f(c - x_p)
 *                               (resolved chain replaces the centre of mass);
 *   a_chain[3k..], pot_chain[k]: sum_p m_p f(x_p - x_k) (perturbers on members);
 *   out8[0..3]  corr = (1/M) sum_k m_k a_chain[k]   (Eq. 3),
 *   out8[3..6]  sub  = sum_p m_p f(x_p - c), the perturbers' direct terms on
 *               the centre-of-mass particle that the tree force contains,
 *   out8[6]     sum_k m_k pot_chain[k] / M, out8[7] = sum_p -m_p / |x_p - c|,
 *   out8[8..11] c, out8[11] M   (out8 holds 12 doubles).
 * f(r) = r / |r|^3; potentials are -m/|r|. Sums run in a fixed order.
 * n_pert may be 0 (then a_pert/pot_pert/pert_* may be NULL). */
rv_status rv_perturber_forces(rv_ctx *ctx, int32_t n_ch, const double *chain_m, const double *chain_x,
                              int32_t n_pert, const double *pert_m, const double *pert_x, double *a_pert,
                              double *pot_pert, double *a_chain, double *pot_chain, double *out8,
                              void *stream);

/* A system advanced by rv_kdk_step: n stars (device FP32, caller order),
 * split into n_members independent members (galaxy realisations that never
 * interact) stored one after another: member k owns stars
 * [member_offsets[k], member_offsets[k+1]) (host int64 [n_members + 1],
 * offsets[0] = 0, offsets[n_members] = n; n_members <= 1 with
 * member_offsets = NULL means one member of all n stars; at most 512
 * members). Each member has its own tree and, if n_chain > 0, n_chains
 * chains (several distant SMBHs: the paper's outlook, Sect. 7) of n_chain
 * members each (device FP64, chain-major and member by member:
 * chain_m[n_members n_chains n_chain], chain_x/v/a[3 ...], chain_pot[...];
 * at most 2048 chain members and 512 chains in total). Every chain's centre
 * of mass is an unsoftened particle of its member's tree; the chains of one
 * member feel each other through these. Perturbers of a chain (stars of its own
 * member): pert_mode 1 = FP32 squared distance to the chain centre below
 * pert_radius^2 (ascending index), 2 = the pert_k nearest (ties by lower
 * index), 3 = the tidal criterion of Eq. 2 with r_crit = pert_radius and
 * gamma_crit = pert_gamma (see rv_select_perturbers_tidal); at most
 * min(5000, 65536 / n_members) per member (overflow of a radius or tidal
 * search is reported by rv_sync_status as RV_E_WORKSPACE).
 * chain_quad: 0 = the stars that are not perturbers feel each chain as its
 * centre-of-mass point mass (Sect. 2 as written); 1 = they also feel the
 * chain's traceless quadrupole about its centre of mass, Q_ab = sum_k m_k
 * (3 d_a d_b - |d|^2 delta_ab), d = x_k - centre, with the cells' expansion
 * (Sect. 1; unsoftened, FP32). Perturbers never get it: they feel the
 * resolved members (FP64) as before. (Without it, the stars around a pair of
 * SMBHs 0.01 apart miss 1e-3 in their force out to r ~ 0.15.) The quadrupole
 * acts on the stars only: the chain members' forces are those of
 * chain_quad = 0. Chains of one member have no quadrupole. */
typedef struct {
    int64_t n;
    float *x, *y, *z, *vx, *vy, *vz;
    const float *m;
    float *ax, *ay, *az, *pot; /* forces at the current positions */
    int32_t n_chain;
    double *chain_m, *chain_x, *chain_v, *chain_a, *chain_pot;
    int32_t pert_mode;
    float pert_radius;
    int32_t pert_k;
    int32_t n_members;
    const int64_t *member_offsets;
    float pert_gamma;
    int32_t n_chains;  /* chains per member (0 or 1: one); chain c belongs to member c / n_chains */
    int32_t chain_quad;
} rv_system;

/* One full force evaluation of a system: tree build, perturber selection,
 * tree forces with the chain's centre of mass as an unsoftened extra
 * particle, FP64 perturber coupling, and the hand-off of the chain (member
 * accelerations = mutual unsoftened FP64 + perturbers + tree force on the
 * centre of mass minus the perturbers' direct terms, Sect. 2). Writes
 * sys->ax..pot and chain_a, chain_pot. */
rv_status rv_system_forces(rv_ctx *ctx, rv_system *sys, void *stream);

/* nsteps kick-drift-kick steps of size dt (global step): v += a dt/2;
 * x += v dt; rv_system_forces; v += a dt/2. Stars in FP32, chain members in
 * FP64. sys->a* must hold the forces at the starting positions (call
 * rv_system_forces once first). */
rv_status rv_kdk_step(rv_ctx *ctx, rv_system *sys, double dt, int32_t nsteps, void *stream);

/* Like rv_kdk_step, but the step (and, if energy_out is not NULL, the
 * rv_energy reduction into device energy_out[10 n_members] after it) is
 * captured once into a CUDA graph and replayed nsteps times: no host work
 * per step. The graph is rebuilt when the system's pointers, offsets, dt or
 * energy_out change; rebuilding first runs rv_system_forces once (forces at
 * the current positions, as the step expects). `stream` must be a created
 * stream (not the legacy or per-thread default stream): RV_E_INVAL
 * otherwise. */
rv_status rv_kdk_step_graph(rv_ctx *ctx, rv_system *sys, double dt, int32_t nsteps, double *energy_out,
                            void *stream);

/* Perturber pull on the chain members for the chain integrator's own force
 * evaluations (Sect. 2: inside its substeps the chain integrator needs the
 * perturbers' forces many times, with the perturbers' positions predicted to
 * first order). Uses the perturber sets of the last rv_system_forces on this
 * system and the stars' current positions and velocities:
 *   x_p(dt) = x_p + v_p dt   (FP64, one rounding per operation),
 *   a_k = sum_p m_p (x_p(dt) - x_k) / |x_p(dt) - x_k|^3,  pot_k = -sum_p m_p / |..|
 * (unsoftened FP64, a fixed summation order) for the chain members at
 * chain_x (device FP64, member-major [3 n_members n_chain], the same frame as
 * the stars). Writes device a_chain[3 n_members n_chain] and, if not NULL,
 * pot_chain[n_members n_chain]. RV_E_NOTBUILT before a force pass of the
 * system. */
rv_status rv_chain_perturber_forces(rv_ctx *ctx, const rv_system *sys, double dt, const double *chain_x,
                                    double *a_chain, double *pot_chain, void *stream);

/* Individual hierarchical block time steps (Sect. 2: the tree code advances
 * its particles on a hierarchy of time-step levels), kick-drift-kick form.
 * Star i is on level level[i] (device int8 [n], 0..max_level), step
 * dt_max / 2^level; the substep is dt_min = dt_max / 2^max_level. A substep
 * drifts all stars and the chain by dt_min; the stars whose step ends then are
 * active: the tree is rebuilt from all stars and only the walk groups holding
 * an active star are walked; active stars get their closing half kick, a new
 * level when adapt = 1 (dt = min(tau_acc sqrt(eps / |a|), tau_vel eps / |v|),
 * level = the smallest l with dt_max 2^-l <= dt, capped at max_level, in FP64;
 * a coarser level only where its step boundary falls on this substep), and the
 * opening half kick of their next step. Chain members move on the finest
 * level (a kick of dt_min per substep). With every level 0 and max_level 0 this
 * is rv_kdk_step. The system's ax..pot hold each star's force of its last
 * active substep. */
typedef struct {
    double dt_max;      /* step of level 0 */
    int32_t max_level;  /* finest level L, 0..20 */
    float tau_acc, tau_vel, eps;  /* step criteria (Sect. 3 uses 0.3 for stars) */
    int32_t adapt;      /* 1: levels follow the criteria; 0: levels stay as given */
    int8_t *level;      /* device int8 [n], in/out */
    int64_t substep;    /* substeps done since rv_block_start (out) */
} rv_blocks;
/* Forces on every star, levels (adapt = 1) and the opening half kicks; substep = 0. */
rv_status rv_block_start(rv_ctx *ctx, rv_system *sys, rv_blocks *b, void *stream);
/* nsub substeps of dt_min (rv_block_start first). */
rv_status rv_block_steps(rv_ctx *ctx, rv_system *sys, rv_blocks *b, int32_t nsub, void *stream);
/* The level rule alone on n stars (device FP32 a and v, caller order) for a
 * host integrator: the stars active at b->substep (all when start != 0, then
 * unconstrained) get the level of the criteria, a coarser one only where its
 * step boundary is at b->substep. Writes b->level. */
rv_status rv_block_levels(rv_ctx *ctx, int64_t n, const float *ax, const float *ay, const float *az,
                          const float *vx, const float *vy, const float *vz, rv_blocks *b, int32_t start,
                          void *stream);
/* Active star updates (forces used by a kick) since rv_block_start; synchronises `stream`. */
rv_status rv_block_count(rv_ctx *ctx, int64_t *active_updates, void *stream);

/* FP64 totals of each member of a system, written to device out[10 k ..] for
 * member k: E_kin, E_pot, E_tot, P (3), L (3), M. Stars: sum m v^2/2,
 * sum m phi/2, sum m v, sum m x cross v; chain members added in FP64 with
 * their potential chain_pot. Deterministic (fixed reduction order). */
rv_status rv_energy(rv_ctx *ctx, const rv_system *sys, double *out, void *stream);

/* Perturber selection on its own (see rv_system): writes ascending indices
 * to device idx[cap] and the count to device count[1]. mode 1 radius, 2 k
 * nearest. centre is a host FP32 point. A radius selection longer than cap
 * is truncated and reported as RV_E_WORKSPACE by rv_sync_status. */
rv_status rv_select_perturbers(rv_ctx *ctx, int64_t n, const float *x, const float *y, const float *z,
                               const float centre[3], int32_t mode, float radius, int32_t k, int32_t cap,
                               int32_t *idx, int32_t *count, void *stream);

/* The chain's start radius (Eq. 1): r_chain,0 = max(alpha r_infl, beta eps)
 * with r_infl = min(r(<2 M_bh), G M_bh / sigma^2) around `centre` (host
 * FP32, the SMBH), sigma the velocity dispersion of the n_sigma (Sect. 2: 50)
 * nearest stars. Stars (device FP32, caller order) in ascending FP32 squared
 * distance, ties by index; r(<2 M_bh) = the distance of the star at which
 * the FP64 running mass in that order first reaches 2 m_bh (infinity if
 * never); sigma = sqrt(sum |v - <v>|^2 / (3 k)) over the k = min(n_sigma, n)
 * nearest, FP64 sums in distance order. Writes host out[5] = r(<2 M_bh),
 * sigma, G M_bh / sigma^2, r_infl, r_chain,0. Synchronises `stream`; the tree
 * must be rebuilt afterwards (shared sort buffers). */
rv_status rv_chain_start_radius(rv_ctx *ctx, int64_t n, const float *x, const float *y, const float *z,
                                const float *vx, const float *vy, const float *vz, const float *m,
                                const float centre[3], double m_bh, int32_t n_sigma, double alpha, double beta,
                                double eps, double out[5], void *stream);

/* Tidal perturber search (Eq. 2): star j (device FP32 x, y, z, m [n]) perturbs
 * a chain of total mass m_chain centred at `centre` (host FP32) when
 *   r_j < (2 m_j / (gamma_crit m_chain))^(1/3) r_crit.
 * Decided without a cube root, in FP64 with one rounding per operation on the
 * FP32 squared distance d2 (as in the radius search):
 *   (d2 d2) d2 < (q q) rc6,  q = (2 m_j) / (gamma_crit m_chain),
 *   rc6 = (rc2 rc2) rc2,  rc2 = r_crit r_crit.
 * Ascending indices to device idx[cap], count to device count[1]; more than
 * cap is truncated and reported as RV_E_WORKSPACE by rv_sync_status. */
rv_status rv_select_perturbers_tidal(rv_ctx *ctx, int64_t n, const float *x, const float *y, const float *z,
                                     const float *m, const float centre[3], float m_chain, float gamma_crit,
                                     float r_crit, int32_t cap, int32_t *idx, int32_t *count, void *stream);

/* Absorption into a chain (Eq. 4): the chain's centre of mass c (FP64,
 * members in index order) and radius r_chain, the largest member distance
 * from c (Sect. 2: the chain radius of the last chain step), from device
 * FP64 chain_m[n_ch], chain_x[3 n_ch] (1 <= n_ch <= 250); a star j (device
 * FP32 x, y, z [n], caller order) is absorbed when r_j,CoM < r_chain, decided
 * in FP64 with one rounding per operation on squared distances:
 * d = (double)x_j - c per axis, d2 = (dx dx + dy dy) + dz dz, absorbed iff
 * d2 < max over members of the same d2. Writes the first cap absorbed
 * indices (ascending) to device idx[cap], the untruncated count to device
 * count[1] and, if not NULL, r_chain to device r_chain[1]. The chain's own
 * members should not be among the stars (they are no longer tree particles). */
rv_status rv_chain_absorb(rv_ctx *ctx, int64_t n, const float *x, const float *y, const float *z, int32_t n_ch,
                          const double *chain_m, const double *chain_x, int32_t cap, int32_t *idx, int32_t *count,
                          double *r_chain, void *stream);

/* Escape from a chain (Eq. 5) and the membership rules around it (Sect. 2
 * and Sect. 3), on the host for one chain of n_ch <= 250 members (host FP64
 * m[n_ch], x[3 n_ch], v[3 n_ch]; massive[k] = 1 for an SMBH; designated = the
 * member that is the chain's designated massive particle). With c, v_c the
 * members' centre-of-mass position and velocity, d = x_k - c, u = v_k - v_c:
 * member k escapes when (d.d) > (gamma r_chain0)^2 and (d.u) > 0 (receding),
 * dot products summed (x + y) + z in FP64 with one rounding per operation;
 * while n_absorbing > 0 perturbers are being absorbed (Eq. 4) escapes wait,
 * unless the chain radius exceeds the escape radius by more than 5 %. The
 * chain ends (terminate = 1) when fewer than 2 members remain, or when the
 * designated member escapes and no other massive member remains; if another
 * remains, the most massive one (lowest index on ties) becomes designated.
 * Writes escape[k] (host, 1 = leaves) and *res. No device work. */
typedef struct {
    int32_t escape_count;
    int32_t terminate;
    int32_t designated;
    double r_chain;    /* largest member distance from the centre of mass */
    double r_escape;   /* gamma r_chain0 */
} rv_chain_escape_result;
rv_status rv_chain_escape(int32_t n_ch, const double *m, const double *x, const double *v, const int32_t *massive,
                          int32_t designated, double r_chain0, double gamma, int32_t n_absorbing, int32_t *escape,
                          rv_chain_escape_result *res);

/* ---- Learned cell-force correction (not in the paper, whose tree uses the
 * multipoles alone). A network of 14 features -> 64 -> 64 -> 3 (SiLU;
 * bfloat16 weights and activations, FP32 accumulation on the tensor cores)
 * predicts, for a point at r = x - com from an accepted cell of side s and
 * mass M, (exact softened force of the cell's stars - its monopole +
 * quadrupole force) * |r|^2 / M. Features (16 floats per row, 14 used):
 * r/|r| (3), s/|r|, eps/|r|, Q/(M s^2) (xx, yy, zz, xy, xz, yz), and the
 * octupole term of the cell's acceleration in the output's units (3),
 * (5/2) [3 v - 7 r^ (r^ . v)] / (M |r|^3) with r^ = r/|r| and v = O(., r^, r^),
 * O the cell's traceless third moment about its centre of mass (a leaf's
 * from its stars, an internal cell's from its children's masses and
 * quadrupoles).
 * The parameter block (rv_mlp_param_bytes, device, caller-owned) holds FP32
 * master weights, Adam moments and bfloat16 copies. */
size_t rv_mlp_param_bytes(void);
/* Device scratch rv_mlp_gradient needs for a batch of `batch` rows. */
size_t rv_mlp_scratch_bytes(int64_t batch);
/* Glorot-uniform weights from a SplitMix64 stream of `seed`, zero biases, an
 * unbounded feature box. */
rv_status rv_mlp_init(void *params, uint64_t seed, void *stream);
/* The feature box: the range of features the network was trained on, per
 * feature [lo, hi]. rv_tree_forces_mlp applies no correction to a (group,
 * cell) pair with any used feature outside it (the pair keeps its plain tree
 * force). Fit sets it to the per-feature minimum and maximum of device rows
 * x[n][16] (n >= 1); set copies host lo[16], hi[16] (lo <= hi, +-inf allowed;
 * synchronises `stream`). RV_E_INVAL on bad arguments. */
rv_status rv_mlp_fit_feature_box(void *params, int64_t n, const float *x, void *stream);
rv_status rv_mlp_set_feature_box(void *params, const float *lo, const float *hi, void *stream);
/* y[n][3] = network(x[n][16]) (device FP32), on the tcgen05 tensor cores in
 * tiles of 128 rows (x need not be 16-byte aligned; aligned rows load as
 * float4). A completion wait that times out (after ~1 s) leaves NaN in the
 * rows of that tile. */
rv_status rv_mlp_forward(const void *params, int64_t n, const float *x, float *y, void *stream);
/* FP64 direct summation for a sample of targets: the reference the tree's
 * force error is measured against (Sect. 3/4 compare tree forces with direct
 * summation). All arrays device FP64, caller-owned: bodies x, y, z, m,
 * eps [n] (eps 0: unsoftened), target indices targets[nt] (int64, into
 * 0..n-1), outputs ax, ay, az, pot [nt]:
 *   a_i = sum_{j != i} m_j d / (d.d + e^2)^{3/2}, phi_i = -sum m_j / (d.d + e^2)^{1/2},
 * d = x_j - x_i, G = 1, e = max(eps_i, eps_j) or 0 if either is 0; a pair with
 * d.d + e^2 = 0 adds nothing. A target index outside 0..n-1 gives NaN.
 * scratch: device, at least rv_direct_fp64_scratch_bytes(nt) bytes. Partial
 * sums over source chunks are added in chunk order (deterministic). Plain
 * FP64 sums. Asynchronous on `stream`. RV_E_INVAL on bad arguments,
 * RV_E_WORKSPACE if the scratch is too small. */
size_t rv_direct_fp64_scratch_bytes(int64_t nt);
rv_status rv_direct_fp64(int64_t n, const double *x, const double *y, const double *z, const double *m,
                         const double *eps, int64_t nt, const int64_t *targets, double *ax, double *ay, double *az,
                         double *pot, void *scratch, size_t scratch_bytes, void *stream);

/* Self-test of the bounded completion wait that guards every tensor-core
 * (tcgen05) kernel here (the paper has no counterpart: this checks the failure
 * path without faulting the GPU). One CTA allocates 32 TMEM columns, waits up
 * to limit_cycles (0 .. 2^32) SM clock cycles on an mbarrier that gets its one
 * arrival (arrive = 1) or none (arrive = 0), frees the TMEM and writes
 * gave_up[0] (device int32) = 1 if the wait ran out, else 0. Asynchronous on
 * `stream`; RV_E_INVAL on bad arguments. */
rv_status rv_wait_selftest(int64_t limit_cycles, int32_t arrive, int32_t *gave_up, void *stream);
/* Mean squared error of network(x) against t[n][3] and its gradient with
 * respect to the FP32 parameter vector (grad: device FP32 [5768], ordered W1
 * 16x64, b1, W2 64x64, b2, W3 64x8, b3, row-major; loss: device FP32 [1] or
 * NULL). Sums run in a fixed order. */
rv_status rv_mlp_gradient(const void *params, int64_t n, const float *x, const float *t, float *grad, float *loss,
                          void *scratch, size_t scratch_bytes, void *stream);
/* One Adam step (step >= 1) on the master weights; refreshes the copies. */
rv_status rv_mlp_adam(void *params, const float *grad, int32_t step, float lr, float beta1, float beta2,
                      float adam_eps, void *stream);
/* Training of the network on device rows in one call: `steps` Adam steps
 * (Kingma & Ba; Adam step numbers step0, step0 + 1, ...) on minibatches of
 * `batch` rows drawn with replacement: row i of step k is row
 * floor(h n / 2^64) of (x, t), h = SplitMix64(seed + k batch + i) (64-bit
 * wrap-around; SplitMix64 of Steele, Lea & Flood 2014), each step the mean
 * squared error and its gradient as rv_mlp_gradient computes them. With
 * fit_box = 1 the feature box becomes the range of all n rows afterwards
 * (rv_mlp_fit_feature_box). x: device [n][16], 16-byte aligned; t: device
 * [n][3]. */
typedef struct {
    int64_t n;
    const float *x, *t;
    int32_t steps, batch;
    int32_t step0;
    float lr, beta1, beta2, adam_eps;
    uint64_t seed;
    int32_t fit_box;
} rv_mlp_train_cfg;
/* Device scratch rv_mlp_train needs for minibatches of `batch` rows (0 if batch < 1). */
size_t rv_mlp_train_scratch_bytes(int32_t batch);
/* losses: device FP32 [steps] receiving each step's loss, or NULL. All work is
 * enqueued on `stream` (no host synchronisation). RV_E_INVAL on bad arguments,
 * RV_E_WORKSPACE if the scratch is too small. */
rv_status rv_mlp_train(void *params, const rv_mlp_train_cfg *cfg, float *losses, void *scratch,
                       size_t scratch_bytes, void *stream);
/* The network's whole state (master weights, Adam moments, bfloat16 copies,
 * feature box) to and from a host byte buffer of rv_mlp_state_bytes(): a
 * 64-byte header (magic "rvmlp", version 1, the layer sizes, the block size)
 * then the parameter block. Both synchronise `stream`. rv_mlp_load returns
 * RV_E_INVAL for a buffer that is too small or whose header does not match
 * this library's network. */
size_t rv_mlp_state_bytes(void);
rv_status rv_mlp_save(const void *params, void *host, size_t bytes, void *stream);
rv_status rv_mlp_load(void *params, const void *host, size_t bytes, void *stream);
/* Training samples from the last tree: n_samples random stars (SplitMix64 of
 * seed), each paired with a cell chosen uniformly among the cells its own
 * walk accepts at theta (its box: its grid cell). Writes features x[n][16],
 * targets t[n][3] (exact residual, FP32) and pairs[2n] = (sorted star slot,
 * cell index; cell -1 if none accepted, then x, t are zero). */
rv_status rv_mlp_samples(rv_ctx *ctx, float theta, float eps_star, int64_t n_samples, uint64_t seed, float *x,
                         float *t, int32_t *pairs, void *stream);
/* Tree forces at theta (as rv_tree_forces, no extra particles) plus the
 * learned correction: the walk records every (group, cell) pair accepted at
 * theta that a walk at theta_rec (< theta) would open, into device pairs[2
 * pair_cap] with the count in npairs[1]; the network evaluates each pair at
 * the group's geometric centre and adds the correction (device scratch
 * gcorr[3 n]) to every star of the group. A pair whose features lie outside
 * the network's feature box gets no correction (the plain tree). Synchronises
 * `stream` once. The network runs as rv_mlp_forward does; a timed-out
 * completion wait is reported as RV_E_TIMEOUT by rv_sync_status. */
rv_status rv_tree_forces_mlp(rv_ctx *ctx, const void *params, float theta, float theta_rec, float eps_star,
                             float *ax, float *ay, float *az, float *pot, int32_t *pairs, int32_t pair_cap,
                             int32_t *npairs, float *gcorr, void *stream);

/* Radius perturber search that allocates nothing and needs no context.
 * (The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- e.g. a chain integrator that looks for
 * perturbers from inside its own step or from a host callback, or a host
 * application that forbids device allocation after start-up.)
 *
 * Same indices as rv_select_perturbers(mode 1): the stars whose FP32
 * squared distance to centre, ((dx*dx + dy*dy) + dz*dz) with every operation
 * rounded once, is below radius*radius (one FP32 product), in ascending
 * order; the first min(total, cap) of them are written to device idx[cap].
 * Device count[1] receives the untruncated total: count > cap means the
 * search was truncated to its first cap indices.
 *
 * Scratch: a fixed 32 KiB device array inside librv (one count per block of
 * 2048 stars), held by every GPU that loads the library until the process
 * exits. Limit: n <= 16,777,216 stars; larger n returns RV_E_TOO_LARGE
 * without launching anything. The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. Every call overwrites the
 * part of the array it uses before reading it, so no clearing is needed, but
 * all calls share the one array: calls whose GPU work overlaps (different
 * streams, or other host threads) race and may return wrong results. x, y, z
 * are device FP32 [n]; centre is a host FP32 point; stream as elsewhere.
 * Returns RV_E_CUDA if one of its own launches fails (an error left by
 * earlier, unrelated work is neither reported nor cleared). The cached
 * address does not survive cudaDeviceReset: do not reset a device while this
 * library is loaded. */
rv_status rv_select_radius_static(int64_t n, const float *x, const float *y, const float *z,
                                  const float centre[3], float radius, int32_t cap, int32_t *idx,
                                  int32_t *count, void *stream);

/* Read-only views of the last tree (device pointers into the workspace,
 * valid until the next build). Synchronises `stream` to read the sizes.
 *   keys    uint64 [n] sorted keys;     perm int32 [n] sorted slot -> caller index
 *   pos     float4 [n] sorted (x, y, z, m)
 *   cbox    int4 [ncell] (ox, oy, oz, level) integer-grid box origin, side 2^(21-level)
 *   clink   int4 [ncell] (child first, n children, first star, star count)
 *   cmom    float4 [3 ncell] (M, com x, y, z), (Qxx, Qyy, Qzz, Qxy), (Qxz, Qyz, 0, 0)
 *   cparent int32 [ncell]
 *   groups  int32 [ngroup][8] (first star, count, box lo x, y, z, box hi x, y, z): runs of
 *           `group` consecutive stars per member, box = tightest integer-grid box of their cells
 *   bounds  double [5] (min x, y, z, L, 2^21/L) */
typedef struct {
    int64_t n, ncell, ngroup;
    const uint64_t *keys;
    const int32_t *perm;
    const float *pos;
    const int32_t *cbox, *clink;
    const float *cmom;
    const int32_t *cparent, *groups;
    const double *bounds;
} rv_tree_view;
rv_status rv_get_tree(rv_ctx *ctx, rv_tree_view *out, void *stream);

/* Interaction counts of the last rv_tree_forces (synchronises `stream`):
 * out[0] = P2P pairs, out[1] = multipole (M2P) pairs, over all targets;
 * out[2] = deepest walk stack (pending child ranges) seen since the context
 * got its workspace. */
rv_status rv_walk_stats(rv_ctx *ctx, int64_t out[3], void *stream);

/* Synchronises `stream` and returns the first error latched by a kernel since
 * the last call (and clears it), else RV_OK. */
rv_status rv_sync_status(rv_ctx *ctx, void *stream);

/* Walk timing: with enable != 0, every later tree-walk launch on this context
 * that is not part of a graph capture records a pair of CUDA events around
 * the walk kernel on its own stream; enabling (or disabling) clears the
 * record. rv_walk_time waits for the recorded launches and returns their
 * summed duration in milliseconds and their number. */
rv_status rv_profile_walk(rv_ctx *ctx, int32_t enable);
rv_status rv_walk_time(rv_ctx *ctx, double *total_ms, int64_t *launches);

/* Number of kernels librv has launched through this context since it was
 * created (host-side count, incremented at each launch). */
int64_t rv_launch_count(const rv_ctx *ctx);

/* Text of the last error on this context ("" if none). Never NULL. */
const char *rv_last_error(const rv_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RV_H */
