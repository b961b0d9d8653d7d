/* The C-ABI used from plain C: argument checks, then two steps of a state in
 * host memory.  Reads grid.bin, z_ifc.bin and state.bin from the working
 * directory (int32 n_cells, n_edges, n_verts, nlev; int32 c2v, c2e, e2c, e2v,
 * v2e, v2c; float64 cell, vertex and edge coordinates / z_ifc / vn, w, rho,
 * exner, theta_v, exner_pr, level-contiguous) and writes the stepped state to
 * out.bin in the same order.  Exit status 0 when every check passed. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "icon_dycore.h"

static int failures = 0;
#define CHECK(cond, what)                                 \
  do {                                                    \
    if (!(cond)) {                                        \
      fprintf(stderr, "FAILED: %s (%s)\n", what, icon_last_error()); \
      ++failures;                                         \
    }                                                     \
  } while (0)

static void* read_n(FILE* f, size_t bytes) {
  void* p = malloc(bytes);
  if (!p || fread(p, 1, bytes, f) != bytes) {
    fprintf(stderr, "short read\n");
    exit(2);
  }
  return p;
}

int main(void) {
  FILE* f = fopen("grid.bin", "rb");
  if (!f) return 2;
  int32_t dims[4];
  if (fread(dims, sizeof dims, 1, f) != 1) return 2;
  const int32_t nc = dims[0], ne = dims[1], nv = dims[2], nlev = dims[3];
  icon_grid_desc_t d;
  memset(&d, 0, sizeof d);
  d.n_cells = nc;
  d.n_edges = ne;
  d.n_verts = nv;
  d.index_base = 0;
  d.sphere_radius = 6.371229e6;
  d.c2v = read_n(f, 3 * (size_t)nc * 4);
  d.c2e = read_n(f, 3 * (size_t)nc * 4);
  d.e2c = read_n(f, 2 * (size_t)ne * 4);
  d.e2v = read_n(f, 2 * (size_t)ne * 4);
  d.v2e = read_n(f, 6 * (size_t)nv * 4);
  d.v2c = read_n(f, 6 * (size_t)nv * 4);
  d.cell_xyz = read_n(f, 3 * (size_t)nc * 8);
  d.vert_xyz = read_n(f, 3 * (size_t)nv * 8);
  d.edge_xyz = read_n(f, 3 * (size_t)ne * 8);
  fclose(f);
  f = fopen("z_ifc.bin", "rb");
  if (!f) return 2;
  double* z_ifc = read_n(f, (size_t)(nlev + 1) * 8);
  fclose(f);
  const size_t ef = (size_t)ne * nlev, cf = (size_t)nc * nlev, ch = (size_t)nc * (nlev + 1);
  f = fopen("state.bin", "rb");
  if (!f) return 2;
  icon_state_t s;
  s.vn = read_n(f, ef * 8);
  s.w = read_n(f, ch * 8);
  s.rho = read_n(f, cf * 8);
  s.exner = read_n(f, cf * 8);
  s.theta_v = read_n(f, cf * 8);
  s.exner_pr = read_n(f, cf * 8);
  fclose(f);

  /* argument checks (nothing on the GPU happens for these) */
  icon_grid_t* g = NULL;
  CHECK(icon_grid_create(NULL, &g) == ICON_ERR_ARG, "NULL grid description rejected");
  CHECK(strlen(icon_last_error()) > 0, "error message set");
  CHECK(icon_grid_destroy(NULL) == ICON_OK, "destroying NULL grid is a no-op");
  CHECK(icon_dycore_destroy(NULL) == ICON_OK, "destroying NULL dycore is a no-op");

  CHECK(icon_grid_create(&d, &g) == ICON_OK && g, "grid created");
  icon_dycore_params_t p;
  icon_dycore_params_default(&p);
  p.dtime = 1800.0;
  p.autotune = 0;
  p.synchronous = 1;
  icon_dycore_t* dy = NULL;
  CHECK(icon_dycore_create(g, 0, z_ifc, &p, &dy) == ICON_ERR_ARG, "nlev = 0 rejected");
  CHECK(icon_dycore_create(g, nlev, z_ifc, &p, &dy) == ICON_OK && dy, "dycore created");
  if (failures) return 1;
  CHECK(icon_dycore_step(dy, NULL) == ICON_ERR_ARG, "NULL state rejected");
  icon_state_t bad = s;
  bad.rho = NULL;
  CHECK(icon_dycore_step(dy, &bad) == ICON_ERR_ARG, "NULL state field rejected");
  int32_t sz[4] = {0, 0, 0, 0};
  CHECK(icon_dycore_sizes(dy, &sz[0], &sz[1], &sz[2], &sz[3]) == ICON_OK && sz[0] == nlev && sz[1] == nc &&
            sz[2] == ne && sz[3] == nv,
        "sizes reported");

  for (int step = 0; step < 2; ++step) CHECK(icon_dycore_step(dy, &s) == ICON_OK, "step with host arrays");

  f = fopen("out.bin", "wb");
  if (!f) return 2;
  fwrite(s.vn, 8, ef, f);
  fwrite(s.w, 8, ch, f);
  fwrite(s.rho, 8, cf, f);
  fwrite(s.exner, 8, cf, f);
  fwrite(s.theta_v, 8, cf, f);
  fwrite(s.exner_pr, 8, cf, f);
  fclose(f);
  CHECK(icon_dycore_destroy(dy) == ICON_OK, "dycore destroyed");
  CHECK(icon_grid_destroy(g) == ICON_OK, "grid destroyed");
  printf("%d failures\n", failures);
  return failures ? 1 : 0;
}
