/* CPU oracle of the traffic microsimulation hot path (Waddell et al., Sec. 6).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded C written from the
 * paper; it shares no code with the CUDA library.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Conventions: arrays are caller-owned and copied at creation; all per-trip
 * outputs are indexed by trip id (vid).  Return codes: 0 ok, -1 invalid
 * argument, -2 out of memory, -4 unreachable destination, -6 bad state.
 */
#ifndef GBT_ORACLE_H
#define GBT_ORACLE_H
#include <stdint.h>

typedef struct {
  int32_t n_nodes, n_links;
  const int32_t *node_x_dm, *node_y_dm;
  const uint8_t *node_control;          /* 0 none, 1 stop, 2 signal */
  const int32_t *signal_offset_ds, *signal_cycle_ds, *signal_green_ds;
  const int32_t *link_from, *link_to;
  const float *link_length_m, *link_speed_mps;
  const uint8_t *link_lanes, *link_class;
} orc_network;

typedef struct {
  int32_t n_trips;
  const int32_t *origin, *dest, *depart_step;
} orc_demand;

typedef struct {
  float dt, veh_len, s_min;
  int32_t n_class;
  const float *v0, *T, *a, *b, *s0;     /* [n_class]; v0 <= 0 -> link speed */
  float mobil_p, mobil_athr, mobil_bsafe, mobil_bias_right;
  float lambda_mand, stop_acquire_m;
  uint64_t seed;
  int32_t cost_mode, loop_routes;
} orc_params;

typedef struct orc_sim orc_sim;

int  orc_create(const orc_network*, const orc_demand*, const orc_params*, orc_sim** out);
void orc_destroy(orc_sim*);
int  orc_route(orc_sim*, const int32_t* link_cost_ds /* NULL = free-flow */);
int  orc_set_routes(orc_sim*, const int32_t* offsets, const int32_t* links);
int  orc_route_size(const orc_sim*, int64_t* n_hops);
int  orc_read_routes(const orc_sim*, int32_t* offsets, int32_t* links);
int  orc_write_state(orc_sim*, const uint8_t* status, const int32_t* link, const int32_t* lane,
                     const int32_t* cursor, const float* x, const float* v);
int  orc_step(orc_sim*, int32_t n_steps);
int  orc_read_state(const orc_sim*, uint8_t* status, int32_t* link, int32_t* lane, int32_t* cursor,
                    float* x, float* v, int32_t* insert_step, int32_t* arrive_step, int8_t* lane_change);
int  orc_occupancy(const orc_sim*, int32_t* lane_start /* [n_lanes+1] */, int32_t* sorted_vid);
int  orc_n_lanes(const orc_sim*);
int  orc_counters(const orc_sim*, int64_t out[9]);
int  orc_node_holder(const orc_sim*, int32_t* holder);

/* calibration (not in the paper): route progress every obs_every steps, and the
 * gradient of the squared progress error with respect to the IDM parameters of every
 * class (v0, T, a, b, s0), discrete decisions held fixed; binary64 reverse sweep */
int  orc_observe(orc_sim*, int32_t n_steps, int32_t obs_every, double* progress);
int  orc_adjoint(orc_sim*, int32_t n_steps, int32_t obs_every, const double* target, double* grad, double* loss);
int  orc_replay_loss(const orc_sim*, const double* v0, const double* T, const double* a, const double* b,
                     const double* s0, double* loss);
int  orc_set_class_params(orc_sim*, const float* v0, const float* T, const float* a, const float* b, const float* s0);
/* test helpers: a recorded run without the reverse sweep, and the digest of the
 * discrete decisions of the last recorded run (equal digests: no discrete event flipped) */
int  orc_record(orc_sim*, int32_t n_steps);
int  orc_tape_digest(const orc_sim*, uint64_t* digest, int64_t* n_rec, uint64_t* step_digest);

/* measured outputs (flags: 1 fuel and CO per trip, Eq. 8-9; 2 link traversal times,
 * Sec. 6.3.1; 4 per-edge samples, Sec. 6.4), cleared whenever the run restarts */
int  orc_set_outputs(orc_sim*, uint32_t flags, int32_t sample_every, int32_t per_window, int32_t max_windows);
int  orc_reset_outputs(orc_sim*);
int  orc_read_emissions(const orc_sim*, double* fuel_ml, double* co_g);
int  orc_read_link_times(const orc_sim*, int64_t* sum_steps, int32_t* n_exits);
int  orc_read_edge_samples(const orc_sim*, double* util, double* speed, int32_t* n_samples);
/* vehicle types (Sec. 6.3.5): per type length, acceleration scale, maximum speed */
int  orc_set_vehicle_types(orc_sim*, int32_t n, const float* length, const float* accel_scale,
                           const float* max_speed, const uint8_t* trip_type);
/* iterative decaying route equilibrium (Sec. 6.3.1) */
int  orc_measured_costs(const orc_sim*, const int32_t* prev_cost_ds, int32_t* cost_ds, double* gap);
int  orc_reroute(orc_sim*, const int32_t* link_cost_ds, uint32_t fraction_q16, uint32_t round);
int  orc_equilibrium(orc_sim*, int32_t n_iter, const uint32_t* fractions_q16, int32_t n_steps,
                     int32_t* cost_out, double* gap);

/* static user equilibrium (Sec. 5.2, Eq. 6) by Frank-Wolfe on BPR times (Eq. 3) */
int  orc_assign_static(orc_sim*, const double* capacity, double alpha, int32_t beta, int32_t max_iter,
                       int32_t bisect_iter, double* flow, double* time, double* gap, double* step,
                       double* objective);
int  orc_aon(orc_sim*, const int32_t* cost, double* flow);

/* building blocks exposed for the pin tests */
int   orc_reroute_selected(uint64_t seed, int32_t vid, uint32_t round, uint32_t fraction_q16);
float orc_co_rate(float v);
float orc_fuel_rate(float v, float a);
float orc_idm(float a, float b, float T, float s0, float v0, float s_min,
              float s, float v, float v_lead, int has_leader);
void  orc_ballistic(float x, float v, float acc, float dt, float* x_out, float* v_out);
int32_t orc_link_cost(float length_m, float speed_mps, int lanes, int mode);
int   orc_sssp(int32_t n_nodes, int32_t n_links, const int32_t* from, const int32_t* to,
               const int32_t* cost, int32_t origin, int64_t* dist);
uint32_t orc_mand_index(uint64_t seed, int32_t vid, int32_t hop);
float orc_mand_tau(int k);
int   orc_turn(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy);
int   orc_signal_green(int64_t t, int32_t dt_ds, int32_t offset, int32_t cycle, int32_t green, int ew);

#endif
