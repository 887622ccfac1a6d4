/* Oracle-internal: the base planner's footprints and visibility graph
 * (test infrastructure only; see plan2d.cpp). */
#ifndef CEM_ORACLE_PLAN2D_H
#define CEM_ORACLE_PLAN2D_H
#include <stdint.h>

#include "oracle.h"

struct Footprint {
  int n;
  double nx[OR_MAX_SLAB], ny[OR_MAX_SLAB], lo[OR_MAX_SLAB], hi[OR_MAX_SLAB];
};

struct BaseGraph {
  int n_obs;
  Footprint grown[OR_MAX_GEOM], bare[OR_MAX_GEOM];
  int nc;
  double cx[OR_MAX_CORNERS], cy[OR_MAX_CORNERS];
  uint64_t vis[OR_MAX_CORNERS];
};

void base_graph(const or_scene& s, BaseGraph& G);
/* Waypoints of the A* path from (sx, sy) to (gx, gy): the nodes after the
 * start, ending with the goal; returns their number (<= cap). */
int plan_path(const BaseGraph& G, double sx, double sy, double gx, double gy, double* wx, double* wy, int cap);
bool footprint_contains(const Footprint& f, double x, double y);
bool segment_enters(const Footprint& f, double ax, double ay, double bx, double by);

#endif
