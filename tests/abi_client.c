/* A plain C99 client of libifilt (host-side entry points only, no GPU needed):
 * the header must compile as C with warnings as errors, and the library must
 * link and answer from C.  Builds a doubly periodic n x n split-square mesh
 * (unit spacing, every square cut along the same diagonal), prepares it for
 * the scalar vertex placement, and prints what the test checks. */
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "ifilt.h"

#define N 6

int main(int argc, char** argv) {
  static double coords[N * N * 2];
  static int32_t tri[2 * N * N * 3];
  int i, j, t = 0;
  const char* path = argc > 1 ? argv[1] : "abi_client.ifmesh";
  for (j = 0; j < N; j++)
    for (i = 0; i < N; i++) {
      coords[2 * (j * N + i)] = i;
      coords[2 * (j * N + i) + 1] = j;
    }
  for (j = 0; j < N; j++)
    for (i = 0; i < N; i++) {
      const int32_t a = j * N + i, b = j * N + (i + 1) % N;
      const int32_t c = ((j + 1) % N) * N + (i + 1) % N, d = ((j + 1) % N) * N + i;
      tri[t++] = a; tri[t++] = b; tri[t++] = c;
      tri[t++] = a; tri[t++] = c; tri[t++] = d;
    }
  ifilt_mesh_desc desc;
  memset(&desc, 0, sizeof desc);
  desc.n_vert = N * N;
  desc.n_tri = 2 * N * N;
  desc.coords = coords;
  desc.tri = tri;
  desc.ocean = NULL;
  desc.geometry = IFILT_GEOM_PLANAR_PERIODIC;
  desc.period_x = N;
  desc.period_y = N;
  desc.placement = IFILT_VERTEX_SCALAR;
  desc.max_order = 2;
  desc.reorder = IFILT_REORDER_RCM;

  ifilt_mesh mesh = NULL;
  if (ifilt_prepare_mesh_host(&desc, &mesh) != IFILT_OK) {
    printf("prepare failed: %s\n", ifilt_last_error());
    return 1;
  }
  ifilt_mesh_info_t info;
  if (ifilt_mesh_info(mesh, &info) != IFILT_OK) return 2;
  printf("rows %d nnz_k %lld nnz_g2 %lld\n", info.n_rows, (long long)info.nnz_k, (long long)info.nnz_g2);

  double* kval = malloc(sizeof(double) * (size_t)info.nnz_k);
  double* mass = malloc(sizeof(double) * (size_t)info.n_rows);
  if (!kval || !mass) return 3;
  if (ifilt_mesh_export(mesh, IFILT_EXPORT_K_VAL, kval, sizeof(double) * (size_t)info.nnz_k) != IFILT_OK) return 4;
  if (ifilt_mesh_export(mesh, IFILT_EXPORT_MASS, mass, sizeof(double) * (size_t)info.n_rows) != IFILT_OK) return 5;
  {
    double sum = 0.0, msum = 0.0;
    long long n_unit = 0, n_four = 0;
    int64_t q;
    for (q = 0; q < info.nnz_k; q++) {
      sum += kval[q];
      n_unit += kval[q] == -1.0;
      n_four += kval[q] == 4.0;
    }
    for (q = 0; q < info.n_rows; q++) msum += mass[q];
    printf("k_sum %.17g k_minus_one %lld k_four %lld mass_sum %.17g\n", sum, n_unit, n_four, msum);
  }

  /* an error status and its message */
  if (ifilt_mesh_export(mesh, IFILT_EXPORT_MASS, mass, 8) != IFILT_EINVAL) return 6;
  printf("error message: %s\n", ifilt_last_error()[0] ? "yes" : "no");

  /* cache round trip */
  uint64_t key = 0, key2 = 0;
  if (ifilt_mesh_key(&desc, &key) != IFILT_OK || ifilt_mesh_get_key(mesh, &key2) != IFILT_OK) return 7;
  if (ifilt_mesh_save(mesh, path, IFILT_SAVE_MULTIGRID) != IFILT_OK) {
    printf("save failed: %s\n", ifilt_last_error());
    return 8;
  }
  ifilt_mesh back = NULL;
  if (ifilt_mesh_load_host(path, key, &back) != IFILT_OK) {
    printf("load failed: %s\n", ifilt_last_error());
    return 9;
  }
  ifilt_mesh other = NULL;
  const ifilt_status wrong = ifilt_mesh_load_host(path, key + 1, &other);
  ifilt_multigrid_info mg;
  if (ifilt_mesh_multigrid(back, &mg) != IFILT_OK) return 10;
  printf("key_match %d wrong_key_status %d mg_levels %d\n", key == key2, (int)wrong, mg.n_levels);
  printf("version %s\n", ifilt_version());
  printf("layout desc %zu %zu opts %zu %zu %zu info %zu stats %zu\n", sizeof(ifilt_mesh_desc),
         offsetof(ifilt_mesh_desc, mg_strength), sizeof(ifilt_solve_opts), offsetof(ifilt_solve_opts, err_tol),
         offsetof(ifilt_solve_opts, mg_cycle), sizeof(ifilt_mesh_info_t), sizeof(ifilt_col_stats));
  printf("layout2 item %zu mg %zu server %zu request %zu profile %zu\n", sizeof(ifilt_solve_item),
         sizeof(ifilt_multigrid_info), sizeof(ifilt_server_opts), sizeof(ifilt_request_info),
         sizeof(ifilt_kernel_profile));
  ifilt_release_mesh(back);
  ifilt_release_mesh(mesh);
  ifilt_release_mesh(NULL);
  free(kval);
  free(mass);
  return 0;
}
