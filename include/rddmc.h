/*
 * rddmc.h -- C-ABI of the GB300 (sm_103a) resonant discrete diffusion Monte
 * Carlo library (Smith, Tsang, Bromm & Milosavljevic 2017, "Discrete diffusion
 * Lyman alpha radiative transfer").
 *
 * The problem a caller states (Sec. 2.2, Sec. 2.3): a medium on a Cartesian
 * grid of cells (hydrogen density, temperature, bulk velocity per cell), a
 * discretisation of the comoving frequency x = (nu - nu0)/dnu_D into bins, and
 * a monochromatic source at the domain centre.  The library walks photon
 * packets on the joint (cell, bin) grid with the Fokker-Planck leakage
 * probabilities of Sec. 2.2 until they leave the domain, and tallies the
 * escaping spectrum.
 *
 * Conventions for every function:
 *   - returns an int status: RDDMC_OK (0) or a negative RDDMC_ERR_* code;
 *     never throws, never exits, never prints;
 *   - "host" pointers are read during the call only; "device" pointers are
 *     caller-owned device memory (for example PyTorch tensors) that must stay
 *     valid until the stream work enqueued by the call has finished;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); device work is enqueued on it and the call does not synchronise
 *     unless stated;
 *   - the library allocates no device memory and never frees caller memory;
 *     the grid handle owns host memory only.
 */
#ifndef RDDMC_H
#define RDDMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- statuses */
#define RDDMC_OK 0
#define RDDMC_ERR_ARG -1          /* invalid argument (null, out of range, inconsistent) */
#define RDDMC_ERR_UNSUPPORTED -2  /* valid input the library does not implement */
#define RDDMC_ERR_SIZE -3         /* a caller buffer is smaller than required */
#define RDDMC_ERR_CUDA -4         /* a CUDA runtime call or kernel launch failed */
#define RDDMC_ERR_STEP_LIMIT -5   /* device status: packets aborted by the step watchdog */
#define RDDMC_ERR_TABLE -6        /* the table buffer was not filled for this grid */
#define RDDMC_ERR_TIMEOUT -7      /* device status: a bounded wait of a tensor-core product ran out */

/* ------------------------------------------------------------- enumerations */
#define RDDMC_GEOM_SLAB_1D 1      /* slab |z| <= R, one spatial axis */
#define RDDMC_GEOM_CART_3D 3      /* cube [-R,R]^3 of Cartesian cells */

#define RDDMC_MODE_DDMC 0         /* DDMC in every state (Sec. 3.2 test problems) */
#define RDDMC_MODE_HYBRID 1       /* thin states hand off to continuous MC (Sec. 5.1-5.2) */

#define RDDMC_DUST_PROBABILISTIC 0 /* dust absorption as a competing process (Sec. 2.6) */
#define RDDMC_DUST_WEIGHTS 1       /* dust absorption by packet weights (Sec. 2.6) */

#define RDDMC_LAYOUT_DEDUP 0      /* one row block per class of identical cells */
#define RDDMC_LAYOUT_DENSE 1      /* one row block per cell */

/*
 * Grid description (host data, copied by rddmc_build_grid).
 *   geometry   RDDMC_GEOM_SLAB_1D or RDDMC_GEOM_CART_3D.
 *   n[3]       cells per axis; a slab uses n[0] and requires n[1] = n[2] = 1.
 *              Cell index c = i0 + n0*(i1 + n1*i2); cubic domain [-R, R]^d with
 *              uniform widths dz_a = 2R/n[a] (Sec. 2.2, eq. z-leakage).
 *   nbins      number J of frequency bins (>= 1, <= 65535).
 *   layout     RDDMC_LAYOUT_DEDUP or RDDMC_LAYOUT_DENSE (table organisation).
 *   R          half-width of the domain (length unit of the problem).
 *   tau0       line-centre optical depth k0 R at unit density (k_x = k0 H(a,x),
 *              Sec. 2.2); a cell's k0 is tau0/R times its n_rel.
 *   T          gas temperature in K (isothermal; sets a = 4.702e-4 T4^-1/2 and
 *              v_th = 12.85 T4^1/2 km/s, Sec. 2.1).
 *   freq_edges host, nbins+1 strictly increasing comoving x edges (FP64).  Moving
 *              media (v_kms != NULL) require uniform bins.
 *   n_rel      host, ncell relative densities >= 0 (FP64), or NULL for 1.
 *   v_kms      host, 3*ncell bulk velocities in km/s (xyz per cell, FP64), or NULL.
 *   mask       host, ncell bytes: 1 medium, 0 vacuum (a packet entering a vacuum
 *              cell escapes), or NULL for all medium.
 */
typedef struct rddmc_grid_desc {
    int32_t geometry;
    int32_t n[3];
    int32_t nbins;
    int32_t layout;
    double R;
    double tau0;
    double T;
    const double* freq_edges;
    const double* n_rel;
    const double* v_kms;
    const uint8_t* mask;
} rddmc_grid_desc;

/*
 * Leakage parameters (Sec. 2.5, Sec. 5.1).
 *   tau_ddmc  thick threshold on tau_ij = k_ij dz (paper suggests 5).
 *   lambda    extrapolation distance of the boundary coefficient (0.7104).
 *   f_mu      flux directionality factor of eq. velocity-shift (1/2 isotropic).
 *   mode      RDDMC_MODE_DDMC or RDDMC_MODE_HYBRID.
 *   dust_abs, dust_scat  grey dust (Sec. 2.6, the probabilistic method):
 *             absorption and scattering optical depths k_a R and k_s R at
 *             unit density (scaled by each cell's n_rel; >= 0).  Scattering
 *             adds k_s to every k_ij of the leakage coefficients; absorption
 *             is one more competing process, the last outcome of every
 *             state's categorical draw, and an absorbed packet ends (counted
 *             in rddmc_tallies.absorbed).  dust_abs > 0 requires DDMC mode.
 *   dust_method RDDMC_DUST_PROBABILISTIC (0, above) or RDDMC_DUST_WEIGHTS (1,
 *             the continuous method): no absorption outcome; each transition
 *             out of state s multiplies the packet weight by K_s/(K_s + k_a),
 *             the expected attenuation exp(-k_a dl) over its dwell, packets
 *             below weight 1e-10 are eliminated (counted absorbed) and escapes
 *             carry their weight (rddmc_tallies.escaped_weight,
 *             rddmc_read_escape_weights).  The time-dependent walk attenuates
 *             by exp(-k_a l) over each path l and reports weighted estimates.
 */
typedef struct rddmc_leak_params {
    double tau_ddmc;
    double lambda;
    double f_mu;
    int32_t mode;
    int32_t dust_method;
    double dust_abs;
    double dust_scat;
} rddmc_leak_params;

/*
 * Run options of one rddmc_launch_packets call.
 *   seed          Philox4x32-10 key (see the stream contract below).
 *   n_packets     packets with ids [0, n_packets), n_packets < 2^63.
 *   max_steps     watchdog: a packet about to take transition max_steps+1 is
 *                 aborted and counted (0 = 2^62).
 *   steps_per_launch  time slice: each packet advances at most this many
 *                 transitions in this call and its state is saved to the state
 *                 buffer; a later call with resume = 1 continues it.  0 = run
 *                 every packet to escape or abort.  Must be a multiple of 4.
 *   resume        0: every packet starts at the source (state buffer is only
 *                 written); 1: continue the packets saved by a previous call on
 *                 the same state buffer, grid, seed and n_packets.
 *   ctas_per_sm, threads_per_cta, chunk  launch schedule (0 = library default):
 *                 persistent grid of ctas_per_sm * #SM CTAs of threads_per_cta
 *                 threads (a multiple of 32, at most 256); `chunk` transitions
 *                 (multiple of 4) between warp refills.
 *   table_in_smem 1: stage the fast row heads in shared memory when they fit;
 *                 0: gather them from global memory (L1/L2).
 *   time_slice_us wall-time slice (0 = none): a thread that reaches a chunk
 *                 boundary more than this many microseconds after its CTA
 *                 started saves its packet and takes no new one.  Needs saved
 *                 states (steps_per_launch > 0, resume = 1 or a proposal).
 *                 Results do not depend on where packets are cut.  When states
 *                 are saved and resume = 0, every packet is first marked as not
 *                 started, so packets a sliced call never reached start in a
 *                 later call with resume = 1.
 *   proposal      NULL, or a learned exit proposal (rddmc_proposal; 3D grids in
 *                 DDMC mode): packets in a state it serves are parked for
 *                 rddmc_propose instead of walking through their brick.  The
 *                 walk checks at transition counts that are multiples of
 *                 `chunk` (and at emission), so parking does not depend on
 *                 slicing.  Requires steps_per_launch > 0, resume = 1 or
 *                 time_slice_us > 0 so parked states are kept.
 *   redist        NULL, or (hybrid tables only) the device thresholds of eq.
 *                 R_discrete from rddmc_precompute_redistribution: the MC of
 *                 thin states then groups frequency (Sec. 5.3), flying with the
 *                 bin-mean opacity k_j and drawing each scattering's new bin
 *                 from the row of the packet's bin (x uniform in it, a new
 *                 isotropic direction) instead of the atom-velocity sampler.
 */
typedef struct rddmc_run_opts {
    uint64_t seed;
    uint64_t n_packets;
    uint64_t max_steps;
    uint64_t steps_per_launch;
    int32_t resume;
    int32_t ctas_per_sm;
    int32_t threads_per_cta;
    int32_t chunk;
    int32_t table_in_smem;
    int32_t time_slice_us;
    const struct rddmc_proposal* proposal;
    const uint32_t* redist;
} rddmc_run_opts;

/* Buffer sizes for a grid (from rddmc_grid_sizes). */
typedef struct rddmc_sizes {
    uint64_t table_bytes;        /* device table buffer (rows, class map, descriptors) */
    uint64_t tally_bytes;        /* device tally buffer */
    uint64_t state_bytes;        /* device state buffer for the n_packets asked for */
    int32_t n_class;             /* row blocks in the table */
    int32_t row_bytes;           /* 16 (slab) or 32 (3D) */
    int32_t n_outcomes;          /* 4 (slab) or 8 (3D), one more with dust absorption (known after
                                    rddmc_precompute_leakage) */
    int32_t reserved;
} rddmc_sizes;

/* Integer tallies of everything launched since the last reset. */
typedef struct rddmc_tallies {
    uint64_t emitted;      /* packets started at the source */
    uint64_t escaped;      /* packets that left the domain */
    uint64_t aborted;      /* packets stopped by the step watchdog */
    uint64_t steps;        /* DDMC transitions executed */
    uint64_t mc_events;    /* continuous-MC events (scatterings and face crossings) */
    uint64_t conversions;  /* DDMC <-> MC hand-offs */
    uint64_t clamps;       /* Doppler rebins clamped to the frequency grid ends */
    uint64_t event_draws;  /* words taken from the packets' event streams */
    uint64_t proposals;    /* learned exit proposals taken */
    uint64_t proposed_steps; /* DDMC transitions the proposals stood in for (sampled) */
    uint64_t absorbed;     /* packets absorbed by dust (Sec. 2.6), or eliminated below weight 1e-10 */
    double escaped_weight; /* weight method: summed weight of the escaped packets (2^-32 resolution) */
    int32_t status;        /* RDDMC_OK or a device-side error code */
    int32_t nbins;         /* J; the histogram has J + 2 entries */
    int32_t nfaces;        /* 2 (slab) or 6 (3D) */
    int32_t nsb;           /* impact-parameter bins (64) of the surface-brightness histogram */
} rddmc_tallies;

typedef struct rddmc_grid rddmc_grid; /* opaque host handle */

/*
 * Random-stream contract.  key = (seed_lo, seed_hi).  Packet p owns two
 * Philox4x32-10 streams of 32-bit words: transition t uses lane t&3 of
 * Philox(ctr = ((t>>2)_lo, (t>>2)_hi, p_lo, p_hi)); event draw e uses lane e&3
 * of Philox(ctr = ((e>>2)_lo, (e>>2)_hi, p_lo, p_hi | 2^31)).  Event draw 0
 * picks the source cell and bin (bit 31-a: cell along axis a when two cells
 * straddle the centre; bit 28: bin when x0 is a bin edge); a Doppler rebin
 * takes one event draw; a DDMC escape takes five (a point on the exit face:
 * two; the outward direction: mu uniform on (0,1] and the azimuth; x uniform
 * in the bin) in 3D and from a moving slab cell, none from a static slab cell.
 */

/*
 * rddmc_build_grid -- validate a grid description and build the host handle.
 * Groups cells whose leakage rows are provably identical (same density,
 * velocity and neighbour data on every face) into classes when layout is
 * RDDMC_LAYOUT_DEDUP; this is the factoring of space and frequency noted for
 * uniform media in Sec. 2.2.  Host-only: no device memory is touched.
 *   desc  host, grid description (read during the call only).
 *   out   host, receives the handle; release it with rddmc_destroy_grid.
 * Errors: RDDMC_ERR_ARG (nulls, non-increasing edges, negative density, bad
 * counts), RDDMC_ERR_UNSUPPORTED (moving media with non-uniform bins).
 */
int rddmc_build_grid(const rddmc_grid_desc* desc, rddmc_grid** out);

/* Release a handle from rddmc_build_grid (NULL is ignored). */
void rddmc_destroy_grid(rddmc_grid* grid);

/*
 * rddmc_grid_sizes -- byte sizes of the caller-owned device buffers.
 *   n_packets  packet count the state buffer must hold.
 *   out        host, receives the sizes.
 */
int rddmc_grid_sizes(const rddmc_grid* grid, uint64_t n_packets, rddmc_sizes* out);

/*
 * rddmc_precompute_leakage -- fill the device table (FP64 kernel).
 * Per state (cell class i, bin j): the bin-mean opacity
 * k_ij = k0_i (calH(a, x_j+) - calH(a, x_j-)) / dx_j (Sec. 2.2), the spatial
 * leakage coefficients of eq. z-leakage (exterior faces and, in hybrid mode,
 * thin neighbours use the boundary form 2/(3 dz (k dz + 2 lambda)), Sec. 5.1),
 * the frequency leakage coefficients of eq. x-leakage (none beyond the grid
 * ends), and the neighbour opacity over the Doppler-shifted bin
 * (eq. velocity-shift).  The probabilities p_X = k_X / sum k are accumulated in
 * the outcome order (bin-1, bin+1, -e0, +e0[, -e1, +e1, -e2, +e2]) and stored
 * as 32-bit thresholds round-half-even(C * 2^32) saturated at 2^32 - 1.
 *   d_table      device, at least sizes.table_bytes, 256-byte aligned.
 *   table_bytes  its size.
 * Errors: RDDMC_ERR_ARG, RDDMC_ERR_SIZE, RDDMC_ERR_CUDA.
 */
int rddmc_precompute_leakage(rddmc_grid* grid, const rddmc_leak_params* params, void* d_table,
                             size_t table_bytes, void* stream);

/*
 * rddmc_reset_tallies -- zero the device tally buffer (stream-ordered).
 *   d_tallies  device, at least sizes.tally_bytes, 8-byte aligned.
 */
int rddmc_reset_tallies(const rddmc_grid* grid, void* d_tallies, size_t tally_bytes, void* stream);

/*
 * rddmc_launch_packets -- walk packets (Sec. 2.3) with one persistent kernel.
 * Each thread holds one packet: it draws one word of the packet's transition
 * stream per transition, gathers the 8-byte head of its state's row (its two
 * frequency thresholds) and, unless the word falls in a plain frequency move,
 * the full 16/32-byte row, and takes the
 * outcome whose threshold interval holds the word (the categorical form of the
 * competing exponentials of eq. l_min_1/2: the argmin of independent
 * exponentials with rates k_X is X with probability k_X / sum k).  Packets
 * leaving the domain (Sec. 2.3: removed at the boundary) are tallied; finished
 * lanes refill from a global packet cursor one warp at a time.  Tallies are
 * accumulated into d_tallies (call rddmc_reset_tallies first).
 *   d_table    device, filled by rddmc_precompute_leakage for this grid.
 *   opts       host, run options.
 *   d_state    device scratch of sizes.state_bytes for opts->n_packets,
 *              256-byte aligned: packet cursor and per-packet saved state.
 *   d_tallies  device tally buffer.
 * Hybrid mode (RDDMC_MODE_HYBRID, Sec. 5.1-5.2): a leak into a thin neighbour
 * hands the packet to continuous MC at a random point of the face with an
 * isotropic outward direction, a leak into a thin bin at a random point of the
 * cell with an isotropic direction (x uniform in the bin in both cases).  MC
 * packets (FP32) fly with k = k0 H(a,x), scatter coherently in the atom frame
 * (isotropic phase function, no recoil), convert back to DDMC after scattering
 * into a thick bin, and at a face into a thick neighbour convert with
 * probability 2/(tau + 2 lambda) (2/3 + mu) or reflect.  MC events do not count
 * against steps_per_launch; max_steps (1e8 when 0) bounds the events of one MC
 * excursion.
 * Errors: RDDMC_ERR_ARG, RDDMC_ERR_SIZE, RDDMC_ERR_TABLE, RDDMC_ERR_CUDA.  Device-side conditions (watchdog
 * aborts) are reported by rddmc_read_tallies.
 */
int rddmc_launch_packets(const rddmc_grid* grid, const void* d_table, const rddmc_run_opts* opts,
                         void* d_state, size_t state_bytes, void* d_tallies, size_t tally_bytes,
                         void* stream);

/*
 * rddmc_read_tallies -- copy the tallies to the host; synchronises `stream`.
 *   out        host, counters and status.
 *   hist       host, J+2 uint64 (index 0: below the frequency grid, 1..J: bins,
 *              J+1: above) of escaping packets in the observer frame, or NULL.
 *   faces      host, 2 (slab: -z, +z) or 6 (-x,+x,-y,+y,-z,+z) uint64 escape
 *              counts per exterior face direction, or NULL.
 *   sb         host, 64 uint64, or NULL: 3D escapes binned by impact parameter
 *              b = |r x n| of the escaping ray (r the exit point relative to
 *              the domain centre, n the direction), 64 bins over b/R in
 *              [0, 1.28) with larger b in the last bin (angle-averaged radial
 *              surface brightness; directional binning, Sec. 5.4).
 * Returns RDDMC_OK; `out->status` holds RDDMC_ERR_STEP_LIMIT if any packet was
 * aborted.
 */
int rddmc_read_tallies(const rddmc_grid* grid, const void* d_tallies, rddmc_tallies* out, uint64_t* hist,
                       uint64_t* faces, uint64_t* sb, void* stream);

/* Escaped weight per escape-histogram bin (weight method of dust absorption):
 * host, J + 2 doubles, the bins of rddmc_read_tallies' hist.  Synchronises.
 * Errors: RDDMC_ERR_ARG, RDDMC_ERR_CUDA. */
int rddmc_read_escape_weights(const rddmc_grid* grid, const void* d_tallies, double* whist, void* stream);

/*
 * rddmc_table_rows -- expand the device table to one row per state (host), for
 * inspection and parity checks.  Synchronises `stream`.
 *   thr    host, ncell * J * (n_outcomes - 1) uint32 cumulative thresholds
 *          (with dust absorption the last one is where absorption starts).
 *   flags  host, ncell * J uint32 flag words (2-bit action per outcome:
 *          0 move, 1 escape, 2 to MC, 3 move with Doppler rebin; bit 30 moving
 *          cell; bit 31 thin state).
 */
int rddmc_table_rows(const rddmc_grid* grid, const void* d_table, uint32_t* thr, uint32_t* flags, void* stream);

/*
 * rddmc_read_packet_states -- copy saved per-packet states [first, first+count)
 * from a state buffer to the host (checkpoint inspection and sampled parity
 * checks).  Synchronises `stream`.  A state is meaningful once a launch with
 * steps_per_launch > 0 or resume = 1 has processed that packet.
 *   n_packets  the n_packets the state buffer was laid out for.
 *   cell, bin  host, count uint32 each: cell index and frequency bin.
 *   steps      host, count uint64: transitions taken so far.
 *   event_draws host, count uint64: event-stream words taken so far.
 *   status     host, count bytes: 0 not started, 1 in flight, 2 finished.
 * Any output pointer may be NULL.  Errors: RDDMC_ERR_ARG (range), RDDMC_ERR_CUDA.
 */
int rddmc_read_packet_states(const rddmc_grid* grid, const void* d_state, uint64_t n_packets, uint64_t first,
                             uint64_t count, uint32_t* cell, uint32_t* bin, uint64_t* steps, uint64_t* event_draws,
                             uint8_t* status, void* stream);

/* --------------------------------------------- discrete frequency grouping
 * Sec. 5.3, eq. R_discrete: the redistribution function averaged over
 * incoming and outgoing bins, R_{j'->j} = (dx_j dx_j')^-1 iint_{j j'}
 * R(x' -> x) dx dx', with R the angle-averaged redistribution of isotropic
 * coherent scattering without recoil (Appendix A).  Row j' is stored as
 * cumulative probabilities at the interior edges e_1..e_{J-1} (32-bit
 * thresholds, round half to even of C 2^32, saturated at 2^32 - 1): the
 * average over x' in bin j' of the fraction of outgoing frequencies below the
 * edge.  Outgoing frequencies beyond the grid count in the end bins.  The x'
 * average takes n_sub Gauss-Legendre nodes of the incoming bin; the integrals
 * in x and in the atom velocity are FP64 Gauss-Legendre on pieces cut at the
 * kinks of R.  The hybrid walk's MC uses the thresholds when rddmc_run_opts.
 * redist points to them.
 */

/* Bytes of the redistribution buffer: J * (J - 1) uint32 (rounded up to 256);
 * 0 for J < 2. */
uint64_t rddmc_redistribution_bytes(const rddmc_grid* grid);

/* Fill d_redist (device, 4-byte aligned, >= rddmc_redistribution_bytes) with
 * the thresholds of eq. R_discrete.  d_table: the grid's precomputed table
 * (256-byte aligned; its bin edges are read).  A launch reads J - 1
 * thresholds for each of the J bins of its own grid, so the buffer it is given
 * must be the one filled for that grid.  n_sub in [1, 8].  Enqueues one kernel on
 * `stream`.  Errors: RDDMC_ERR_ARG, RDDMC_ERR_SIZE, RDDMC_ERR_TABLE,
 * RDDMC_ERR_UNSUPPORTED (n_sub (J - 1) above 25 600), RDDMC_ERR_CUDA. */
int rddmc_precompute_redistribution(const rddmc_grid* grid, const void* d_table, int n_sub, void* d_redist,
                                    size_t bytes, void* stream);

/* ------------------------------------------------------ time-dependent walk
 * Sec. 2.3 (causality within a time step) and eq. E_estimator (the 'bin' and
 * 'path' estimates of the spectral energy density per cell, bin and step).
 * Every packet is emitted at the source at the start of the first step (a
 * flash) and advanced step by step, one launch per step.  In state s a packet
 * draws a dwell path dl = -ln(xi) / K_s, K_s the sum of the state's leakage
 * coefficients (eq. l_min_1/2: the smallest of the competing exponential
 * lengths is Exp(K_s), whichever process wins), then one transition of the
 * DDMC walk.  A dwell that passes the end of the step leaves the packet in its
 * state until then without leaking; the next step draws a fresh dwell.
 * Lengths and times share one unit, that of the grid's R (c = 1).  DDMC-mode
 * tables only.
 *
 * Streams: transitions and event draws as in the persistent walk; dwell word d
 * of packet p is lane d&3 of Philox4x32-10(key = seed, ctr = (d>>2 low,
 * d>>2 high, p low, p high | 2^30)), xi = (word + 1/2) 2^-32.  The dwell is
 * computed in FP32 and rounded to ticks of 2^-31 of the step (the packet
 * clock and the path tallies are integers).
 */
typedef struct rddmc_time_step {
    uint64_t seed;
    uint64_t n_packets;     /* 1 .. 2^62 - 1 */
    uint64_t max_steps;     /* transitions per packet before it is aborted; 0 = 2^62 */
    double t_begin, t_end;  /* the step [t_n, t_{n+1}], t_end > t_begin */
    int32_t start;          /* 1: every packet starts at the source at t_begin (the first step);
                               0: packets resume from the state buffer */
    int32_t chunk;          /* transitions a thread runs between refills: multiple of 4, 0 = 256 */
    int32_t threads_per_cta; /* multiple of 32, at most 256; 0 = 256 */
    int32_t ctas_per_sm;    /* 0 = occupancy limit */
    int32_t regroup;        /* lanes still walking their packets break off, so that the lanes whose
                               packets reached t_end take new ones, once fewer than this many of a
                               warp's lanes are walking (packets keep their state in registers and
                               continue; results do not change): 0 = library default (8),
                               -1 = never, at most 32 */
    int32_t reserved;       /* 0 */
} rddmc_time_step;

/* Bytes of the state buffer of a time-dependent run of n_packets (the
 * persistent walk's state plus a dwell counter per packet); 0 if n_packets is
 * out of range. */
uint64_t rddmc_time_state_bytes(uint64_t n_packets);

/*
 * rddmc_time_step_launch -- enqueue one time step on `stream` (a memset and
 * one kernel; no synchronisation).
 *   d_state    device, 256-byte aligned, state_bytes >= rddmc_time_state_bytes:
 *              per-packet state, kept between steps (caller-owned; step
 *              `start` = 1 needs no initialisation).
 *   d_tallies  device, the walk's tally buffer (rddmc_sizes.tally_bytes),
 *              accumulated: emitted, escaped, aborted, transitions, event
 *              draws, escape faces and histograms, as rddmc_read_tallies reads.
 *   d_bins     device, ncell * J uint64, accumulated (+=): packets in state
 *              s = cell * J + bin at t_end (the bin estimate).
 *   d_path     device, ncell * J uint64, accumulated (+=): path length spent
 *              in state s during the step, in ticks, 2^31 ticks = t_end -
 *              t_begin (the path estimate).
 *   d_counts   device, 5 uint64, accumulated: packets escaped during the step,
 *              dwell draws, transitions, packets in a state at t_end, packets
 *              absorbed by dust during the step.
 *   d_leak     device, ncell * 2 ndim * 2 doubles, accumulated, or NULL: the
 *              leaks of eq. a_estimator.  Entry (cell * 2 ndim + face) * 2 + io
 *              sums k * dl over the packets that leave the cell through that
 *              face (io = 0; k of the cell at the bin it leaves, escapes
 *              included) or enter it through that face (io = 1; k of the cell
 *              at the bin it enters), dl the dwell that ended in the leak, in
 *              ticks (2^31 ticks = t_end - t_begin) times k in units of 1/R.
 *              Faces in the outcome order -x, +x (-y, +y, -z, +z).  The
 *              acceleration of a cell is proportional to sum over faces of
 *              (out - in) times the face's outward normal.
 *   d_wbins, d_wpath  device, ncell * J doubles each, accumulated; required
 *              with dust by weights (Sec. 2.6), else NULL: the bin estimate
 *              weighted by packet weight at t_end, and the path estimate (in
 *              ticks) weighted by the weight averaged along each path, the
 *              weight falling by exp(-k_a l) over a path l; packets below
 *              weight 1e-10 are eliminated (counted absorbed).  Not together
 *              with d_leak.
 * Errors: RDDMC_ERR_ARG (null or misaligned pointer, a field out of range),
 * RDDMC_ERR_TABLE (table not precomputed), RDDMC_ERR_UNSUPPORTED (hybrid-mode
 * table, or ncell * J >= 2^32), RDDMC_ERR_SIZE (a buffer too small),
 * RDDMC_ERR_CUDA.  A packet that meets an MC hand-off is aborted and sets the
 * unsupported-event status bit of the tallies.
 */
int rddmc_time_step_launch(const rddmc_grid* grid, const void* d_table, const rddmc_time_step* step, void* d_state,
                           size_t state_bytes, void* d_tallies, size_t tally_bytes, uint64_t* d_bins,
                           uint64_t* d_path, uint64_t* d_counts, double* d_leak, double* d_wbins, double* d_wpath,
                           void* stream);

/* ----------------------------------------------------------------- batches
 * Many independent grids ("instances", each built and precomputed as above,
 * DDMC mode, any mix of slabs and 3D grids) walked by one persistent launch.
 * Instance i owns global packet ids [off_i, off_i + n_i) with off_0 = 0 and
 * off_{i+1} = off_i + n_i; its packet p uses the streams of global id off_i + p
 * under the run's seed.  Each instance has its own tally block.
 */
typedef struct rddmc_batch rddmc_batch; /* opaque host handle */

/* Describe a batch.  grids/d_tables/n_packets: n_inst entries each (host
 * arrays; the grids and device tables must outlive the batch).  Errors:
 * RDDMC_ERR_ARG, RDDMC_ERR_TABLE (a table not precomputed),
 * RDDMC_ERR_UNSUPPORTED (hybrid-mode grid). */
int rddmc_batch_create(const rddmc_grid* const* grids, const void* const* d_tables, const uint64_t* n_packets,
                       int n_inst, rddmc_batch** out);
void rddmc_batch_destroy(rddmc_batch* batch);

/* Sizes of the caller buffers: descriptors (device, 256-byte aligned), tallies
 * (device; instance blocks of the single-grid tally layout, back to back),
 * scratch (device, packet cursor), and the total packet count.  Any pointer
 * may be NULL. */
int rddmc_batch_sizes(const rddmc_batch* batch, uint64_t* desc_bytes, uint64_t* tally_bytes,
                      uint64_t* scratch_bytes, uint64_t* total_packets);

/* Copy the instance descriptors to d_desc (synchronises `stream`).
 * trial_fraction in (0, 1]: the share of each instance's packets (at least
 * one) that trial launches run, for the autotuner. */
int rddmc_batch_upload(rddmc_batch* batch, double trial_fraction, void* d_desc, size_t desc_bytes, void* stream);

/* Enqueue one persistent launch over every instance (trial != 0: the trial
 * subsets only).  Only a memset and a kernel launch are enqueued.  opts: seed,
 * max_steps, ctas_per_sm, threads_per_cta, chunk (n_packets is ignored;
 * steps_per_launch and resume must be 0).  Tallies accumulate into d_tallies. */
int rddmc_batch_launch(const rddmc_batch* batch, const void* d_desc, const rddmc_run_opts* opts, int trial,
                       void* d_scratch, size_t scratch_bytes, void* d_tallies, size_t tally_bytes, void* stream);

/* Tallies of instance `inst` (as rddmc_read_tallies; synchronises). */
int rddmc_batch_read_tallies(const rddmc_batch* batch, const void* d_tallies, int inst, rddmc_tallies* out,
                             uint64_t* hist, uint64_t* faces, uint64_t* sb, void* stream);

/* Capture {zero the tallies, zero the cursor, launch the batch} on `stream`
 * (a non-default stream) into a CUDA graph and instantiate it;
 * *graph_exec receives a cudaGraphExec_t.  Replay it with
 * rddmc_batch_graph_launch; free it with rddmc_batch_graph_destroy. */
int rddmc_batch_graph_create(const rddmc_batch* batch, const void* d_desc, const rddmc_run_opts* opts,
                             void* d_scratch, size_t scratch_bytes, void* d_tallies, size_t tally_bytes,
                             void* stream, void** graph_exec);
int rddmc_batch_graph_launch(void* graph_exec, void* stream);
void rddmc_batch_graph_destroy(void* graph_exec);

/* Autotuner: run the trial subsets under every candidate schedule
 * (threads_per_cta 128 or 256, ctas_per_sm at full or one-less occupancy,
 * chunk 64, 256 or 1024), timed with CUDA events, and return the one with the
 * most transitions per second in *best (and the rate in *best_rate, may be
 * NULL).  Each trial packet walks at most 65536 transitions (or
 * base->max_steps if lower): the trial measures throughput on the run's own
 * instances, so choose a trial_fraction that fills the GPU.  *best keeps
 * base->max_steps.  Synchronises `stream` and overwrites d_tallies. */
int rddmc_batch_autotune(const rddmc_batch* batch, const void* d_desc, const rddmc_run_opts* base, void* d_scratch,
                         size_t scratch_bytes, void* d_tallies, size_t tally_bytes, void* stream,
                         rddmc_run_opts* best, double* best_rate);

/* --------------------------------------------------- learned exit proposal
 * A small network predicts where a packet entering a uniform b^3 brick of
 * medium leaves it (exit face and frequency bin, and a log2 bucket of the DDMC
 * transitions it took), so the walk can replace many transitions inside thick
 * regions by one draw.  Not in the paper: trained on first passages the DDMC
 * walk itself generates.
 */

/* Optical depth tau_ij = k_ij dz of every bin of `cell`'s class (host, J floats;
 * synchronises). */
int rddmc_cell_tau(const rddmc_grid* grid, const void* d_table, int64_t cell, float* tau, void* stream);

/* Training tensors filled by rddmc_fp_generate (all device pointers). */
typedef struct rddmc_fp_train {
    void* d_x;              /* bf16 [n x 16] network inputs */
    int32_t* d_ta;          /* [n] exit face * J + exit bin, -1 if the step cap was reached */
    int32_t* d_tb;          /* [n] floor(log2(transitions)), at most 31 */
    const float* d_lk;      /* [L] log10(k0 dz) of each level's medium */
    const float* d_lp;      /* [J] log10 of the bin-mean profile (k_j / k0) */
    const float* d_xc;      /* [J] bin-centre frequencies */
    int32_t* d_tc;          /* [n] exit face * b^2 + exit position, -1 on a cap; may be NULL */
} rddmc_fp_train;

/* First passages through a uniform b^3 brick (1 <= b <= 64), the training data
 * of the learned exit proposal (an extension beyond the paper: a learned
 * stand-in for many DDMC transitions, Sec. 2.3, inside thick regions).
 * Level l uses the rows of the centre (interior) cell of grids[l] (3D, DDMC
 * mode, precomputed in d_tables[l]; all levels share J).  Sample i (packet id
 * p0+i under `seed`) reads event words 0..2: word 0 picks the level
 * (floor(w L / 2^32)), word 1 the start bin jlo[l] + floor(w (jhi[l]-jlo[l]+1)
 * / 2^32), word 2 a brick cell m = floor(w b^3 / 2^32) = i0 + b i1 + b^2 i2,
 * which is folded into the fundamental domain of the cube's symmetry group
 * (each coordinate i -> min(i, b-1-i), then sorted ascending).  Transitions
 * follow the walk's stream contract from (folded cell, start bin) until a
 * spatial move leaves the brick or `cap` transitions are taken.  d_out: 8
 * int32 per sample {level, start bin, folded cell c0 + b c1 + b^2 c2, exit
 * face (0..5: -x,+x,-y,+y,-z,+z; 6 = cap), exit bin, exit position (q1 + b
 * q2: the last cell's coordinates along the two axes other than the exit
 * face's, lower axis first; -1 on a cap), 0, 0}; d_steps: uint64 transitions.
 * train (may be NULL): also write network inputs and targets. */
int rddmc_fp_generate(const rddmc_grid* const* grids, const void* const* d_tables, int L, int b, const int32_t* jlo,
                      const int32_t* jhi, uint64_t seed, uint64_t p0, uint64_t n, uint64_t cap, int32_t* d_out,
                      uint64_t* d_steps, const rddmc_fp_train* train, void* stream);

/* A trained proposal attached to a walk (all arrays on the device).  The grid
 * is cut into bricks of `brick`^3 cells (1 <= brick <= 64) whose boundaries
 * sit at cell indices = offset (mod brick) on every axis: a cell with index i
 * on an axis has brick coordinate (i + (brick - offset) % brick) / brick, and
 * the brick index is c0 + nb0 (c1 + nb1 c2) with nb_a = ceil((n_a +
 * (brick - offset) % brick) / brick); n_bricks must equal nb0 nb1 nb2, the
 * length of d_brick_lk.  Only bricks wholly inside the grid take proposals,
 * and only in their inner cube: cells whose brick-local coordinates all lie in
 * [margin, brick - 1 - margin] (0 <= 2 margin < brick).  The network models
 * the first passage out of that inner cube of side brick - 2 margin; with
 * margin >= 1 on a medium that is uniform over each brick, every cell of the
 * inner cube and all its neighbours share one medium, so the first passage is
 * exactly that of a uniform medium, and the walk takes over in the brick's
 * outer shell (density contrast, Doppler shifts and exterior faces included).
 * Brick B with brick_lk[B] = log10(k0 dz) of its (uniform) medium, or below
 * -1e29 when it is not eligible, serves a packet in its inner cube at bin j
 * when log_tau_lo <= brick_lk[B] + lp[j] <= log_tau_hi.  The walk is Markov in
 * (cell, bin), so a packet may be handed over in any such state: the walk
 * checks once per chunk of transitions (and at emission or resumption) and
 * parks the packet in the queue (count, ids; capacity n_packets). */
typedef struct rddmc_proposal {
    int32_t brick;
    int32_t offset;
    const float* d_brick_lk;
    const float* d_lp;
    const float* d_xc;
    double log_tau_lo, log_tau_hi;
    unsigned long long* d_queue_count;
    unsigned long long* d_queue_pid;
    int32_t n_bricks;
    int32_t margin;
    /* Region mode, for media that vary from cell to cell: n_bricks x 8 floats
     * summarising each brick's inner cube (see rddmc_fp_region); features are
     * taken in the world frame (no symmetry fold or mirror) from the summary,
     * the bin and the packet's own cell.  NULL: uniform bricks (the fold). */
    const float* d_summary;
} rddmc_proposal;

/* Regions of a medium that varies from cell to cell, for training the
 * proposal there (an extension beyond the paper, like the proposal itself).
 * The grid is cut into bricks of `brick` cells per edge (boundaries at cell
 * indices = offset mod brick, brick index axis 0 fastest, partial bricks
 * counted); a brick's region is its inner cube of side brick - 2 margin.
 *   d_bricks    device, n_eligible brick indices the samples start in (bricks
 *               wholly inside the grid, margin >= 1, so regions are interior).
 *   d_bin_off   device, n_eligible + 1 offsets into d_bins.
 *   d_bins      device, the start bins of listed brick k:
 *               d_bins[d_bin_off[k] .. d_bin_off[k+1]).
 *   d_summary   device, 8 floats per lattice brick summarising its region:
 *               log10(k0 dz) at the geometric-mean density, the standard
 *               deviation of log10 n, the slope of log10 n per axis against
 *               the cell position (2l + 1)/r - 1, the mean and rms comoving
 *               shift f_mu (v_c - v_nb).e / v_th over the region's interior
 *               faces, and one unused value. */
typedef struct rddmc_fp_region {
    int32_t brick;
    int32_t offset;
    int32_t margin;
    int32_t n_eligible;
    const int32_t* d_bricks;
    const int32_t* d_bin_off;
    const int32_t* d_bins;
    const float* d_summary;
} rddmc_fp_region;

/* First passages out of regions of the grid's own medium (3D, DDMC mode, no
 * dust): sample i is packet p0 + i under `seed`; event draws 0-2 pick the
 * brick, the start cell of its region (axis 0 fastest) and the start bin from
 * the brick's list; the packet then takes the walk's own transitions (Sec. 2.3,
 * Doppler rebins across faces taking the next event draws) until an outcome
 * would carry it out of the region, which is not made.  d_out (device, 8 int32
 * per sample): brick, start bin, start cell, exit face (6: none within cap
 * transitions), exit bin, exit cell on the face (the other two axes, lower
 * axis first, u + r v with r the region's side), event draws taken by rebins,
 * 0; d_steps (device, u64): transitions taken, the crossing one included.
 * With `train` (its d_lk unused) also the network inputs (world frame, from
 * the region's summary, the start bin and the start cell's density) and the
 * targets: face * J + exit bin, the log2 step bucket, face * r^2 + exit cell
 * (-1 without an exit). */
int rddmc_fp_region_generate(const rddmc_grid* grid, const void* d_table, const rddmc_fp_region* region,
                             uint64_t seed, uint64_t p0, uint64_t n, uint64_t cap, int32_t* d_out, uint64_t* d_steps,
                             const rddmc_fp_train* train, void* stream);

/* Serve the parked packets of a walk with the trained network: features of
 * the packet's cell folded into its brick's fundamental domain, tensor-core
 * forward pass in batches of at most `batch` rows (a multiple of 64; d_work of
 * rddmc_mlp_work_bytes(batch, n_out) plus batch * (16 * 2 + n_out * 4) bytes),
 * one exit (face, bin, step bucket, and the exit cell on the face from head C
 * when nC = 6 (brick - 2 margin)^2, uniform when nC = 0) sampled per packet
 * from its event
 * stream, mapped back to the world frame (and mirrored back for negative
 * frequencies), placed across the exit face of the inner cube (Doppler rebin
 * or escape tally as the face's row says), and the packet set in flight again.  Clears the queue.
 * Reads the queue's count with one synchronisation of `stream`, then enqueues
 * the work on `stream` without waiting for it (work queued after it on the
 * same stream sees its results).
 * Errors: RDDMC_ERR_ARG (null pointers, including the proposal's device
 * buffers; d_table, d_state or d_work not 256-byte aligned, d_tallies not
 * 8-byte aligned; n_packets outside [1, 2^63); head sizes or brick geometry
 * that do not match the grid), RDDMC_ERR_TABLE (table not precomputed),
 * RDDMC_ERR_UNSUPPORTED (not a 3D DDMC grid without dust), RDDMC_ERR_CUDA. */
int rddmc_propose(const rddmc_grid* grid, const void* d_table, const rddmc_proposal* proposal, uint64_t seed,
                  uint64_t n_packets, void* d_state, void* d_tallies, int n_out, int nA, int nB, int nC,
                  const float* d_wf, const void* d_wb, int batch, void* d_work, uint64_t* n_served, void* stream);

/* The network: 16 inputs, three hidden layers of 128 (ReLU), n_out logits (a
 * multiple of 16): head A = logits [0, nA) (softmax over exit face x bin),
 * head B = [nA, nA + nB) (softmax over step buckets), optional head C =
 * [nA + nB, nA + nB + 6 S) (per exit face, a softmax over its S exit cells).  Parameters: FP32
 * master copy and BF16 copy, same layout, rddmc_mlp_param_count(n_out)
 * elements: W1[128x16] b1 W2[128x128] b2 W3[128x128] b3 W4[n_out x 128] b4
 * (row-major W[out][in]).  Matrix products run on tensor cores with BF16
 * inputs and FP32 accumulation: tcgen05.mma with tensor-memory accumulators
 * and TMA-staged operands; batch sizes are multiples of 64. */
uint64_t rddmc_mlp_param_count(int n_out);
uint64_t rddmc_mlp_work_bytes(int batch, int n_out);
int rddmc_mlp_to_bf16(int n_out, const float* d_wf, void* d_wb, void* stream);
/* Logits (FP32 [batch x n_out]) of bf16 inputs d_x [batch x 16]. */
int rddmc_mlp_forward(int n_out, const float* d_wf, const void* d_wb, const void* d_x, int batch, void* d_work,
                      float* d_logits, void* stream);
/* Sum over the batch of the heads' cross-entropies (*d_loss, device) and the
 * gradient of its batch mean with respect to every parameter (FP32, master
 * layout) for targets d_ta (head A; -1 = ignore the row), d_tb (head B) and,
 * when nC = 6 S > 0, d_tc (head C = logits [nA + nB, nA + nB + nC): a
 * softmax over the S logits of slice d_tc / S only; -1 = no head-C term). */
int rddmc_mlp_loss_grad(int n_out, int nA, int nB, int nC, int S, const float* d_wf, const void* d_wb,
                        const void* d_x, const int32_t* d_ta, const int32_t* d_tb, const int32_t* d_tc, int batch,
                        void* d_work, float* d_grad, float* d_loss, void* stream);
/* Synchronise `stream`, then report and clear the network's device status:
 * RDDMC_OK, or RDDMC_ERR_TIMEOUT when a tensor-core product's bounded wait ran
 * out since the last call (its output tile was left unwritten). */
int rddmc_mlp_status(void* stream);
/* One Adam step (bias-corrected, step >= 1) on the master weights; refreshes
 * the BF16 copy. */
int rddmc_mlp_adam(int n_out, float* d_wf, void* d_wb, const float* d_grad, float* d_m, float* d_v, int step, float lr,
                   float beta1, float beta2, float eps, void* stream);

/*
 * rddmc_scatter_samples -- run the walk's FP32 scattering sampler n times at
 * the incoming frequency x_in (incoming direction +z; sample i uses the event
 * stream of packet i under `seed`) and write the outgoing frequencies to
 * d_out (device, n floats).  Their density is the angle-averaged
 * redistribution function R_II-A(x, x_in) of Appendix A.  For checking the
 * sampler; the table must be precomputed in hybrid mode (the sampler's
 * envelope table lives there): RDDMC_ERR_UNSUPPORTED for a DDMC-mode table.
 */
int rddmc_scatter_samples(const rddmc_grid* grid, const void* d_table, double x_in, uint64_t seed, uint64_t n,
                          float* d_out, void* stream);

/*
 * rddmc_gather_probe -- the memory system's rate of random dependent gathers,
 * the access the walk makes once per transition (a row of its leakage table,
 * at an address that depends on the previous row).  The paper has no
 * counterpart: this measures the denominator of the walk's gather roofline.
 * Every thread of a persistent grid (ctas_per_sm CTAs of threads_per_cta
 * threads on each SM; ctas_per_sm = 0, or more than fit, launches as many as
 * fit) follows `chain` links through d_table, each link one row_bytes load
 * whose first word is the next row's index.  With in_smem each CTA first
 * copies the table into shared memory and chases there; otherwise the loads
 * go through L1, and the table's size decides where they are served (L1, L2
 * or HBM).  Time the call with events on `stream`; rate = *gathers / time.
 *   d_table      device, table_bytes, 256-byte aligned, caller-owned; with
 *                fill = 1 this call first writes a single-cycle permutation
 *                of its rows into it (row r -> (a r + c) mod n), which later
 *                calls with fill = 0 may reuse.
 *   table_bytes  row_bytes x n rows, n a power of two, 64 <= n <= 2^32;
 *                at most 200 KiB with in_smem (else RDDMC_ERR_SIZE).
 *   row_bytes    8 or 16.
 *   d_sink       device, one u64 the kernel may write (keeps the loads live).
 *   gathers      host out: the number of loads the launch makes.
 * Returns RDDMC_ERR_ARG for bad arguments, RDDMC_ERR_CUDA for a failed launch.
 */
int rddmc_gather_probe(void* d_table, uint64_t table_bytes, int row_bytes, int in_smem, uint32_t chain,
                       int ctas_per_sm, int threads_per_cta, uint64_t seed, int fill, unsigned long long* d_sink,
                       uint64_t* gathers, void* stream);

/*
 * rddmc_launch_packets_noalloc -- rddmc_launch_packets for callers that cannot
 * allocate device memory.  The paper has no counterpart: this is a deployment
 * variant.  A caller that cannot call cudaMalloc (for example a plug-in inside
 * a host application that owns all device memory and gives the plug-in none,
 * or code that must not trigger the implicit device-wide synchronisation
 * cudaMalloc can cause) has no state buffer to pass.  This entry point keeps
 * the packet cursor and the saved packet states in a fixed array compiled into
 * the library: RDDMC_NOALLOC_SCRATCH_BYTES of device memory that every GPU
 * which loads the library holds until the process exits.  It allocates
 * nothing itself.
 *   Arguments and results are those of rddmc_launch_packets without d_state
 *   and state_bytes.  A run to completion (steps_per_launch = 0, resume = 0)
 *   takes any packet count; time-sliced or resumed runs must fit their
 *   per-packet state in the array (about 1 million packets) and otherwise
 *   get RDDMC_ERR_SIZE.
 *   Argument checks are rddmc_launch_packets' own (one shared routine); a
 *   learned proposal (opts->proposal) gets RDDMC_ERR_UNSUPPORTED, because its
 *   parked packets need a caller-owned state buffer.
 *   Every call looks up the array's device address on the current device
 *   (a host-side query, so the address stays right after a cudaDeviceReset);
 *   the first call on a device also loads the library's device code there,
 *   so make that first call before any stream capture.  All calls share the
 *   array and it keeps the previous call's
 *   contents: the cursor is reset by every launch, and resume = 1 continues the
 *   packets the previous call saved there.  Calls whose work overlaps on the
 *   GPU race on the array and must be serialised by the caller.
 */
#define RDDMC_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int rddmc_launch_packets_noalloc(const rddmc_grid* grid, const void* d_table, const rddmc_run_opts* opts,
                                 void* d_tallies, size_t tally_bytes, void* stream);

/* Human-readable name of a status code (static storage). */
const char* rddmc_status_string(int status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int rddmc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RDDMC_H */
