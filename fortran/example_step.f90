! Minimal use of the icon_dycore module: a host model that already holds the
! grid tables and a level-contiguous state in host memory advances it by
! nsteps steps (the library copies host arrays in and out around each call).
! The grid and state are read from unformatted stream files written by the
! caller: grid.bin (n_cells, n_edges, n_verts, nlev as int32, then c2v, c2e,
! e2c, e2v, v2e, v2c as int32 and cell, vertex, edge coordinates as float64),
! z_ifc.bin and state.bin (vn, w, rho, exner, theta_v, exner_pr).  The state
! after two steps is written to out.bin in the same layout as state.bin.
program example_step
  use, intrinsic :: iso_c_binding
  use icon_dycore
  implicit none
  integer(c_int32_t) :: nc, ne, nv, nlev
  integer(c_int32_t), allocatable, target :: c2v(:), c2e(:), e2c(:), e2v(:), v2e(:), v2c(:)
  real(c_double), allocatable, target :: cxyz(:), vxyz(:), exyz(:), z_ifc(:)
  real(c_double), allocatable, target :: vn(:, :), w(:, :), rho(:, :), exner(:, :), theta(:, :), exner_pr(:, :)
  type(icon_grid_desc_t) :: desc
  type(icon_dycore_params_t) :: params
  type(icon_state_t) :: state
  type(c_ptr) :: grid, dycore
  integer :: u, step, rc

  open(newunit=u, file="grid.bin", access="stream", form="unformatted", status="old")
  read(u) nc, ne, nv, nlev
  allocate(c2v(3 * nc), c2e(3 * nc), e2c(2 * ne), e2v(2 * ne), v2e(6 * nv), v2c(6 * nv))
  allocate(cxyz(3 * nc), vxyz(3 * nv), exyz(3 * ne))
  read(u) c2v, c2e, e2c, e2v, v2e, v2c, cxyz, vxyz, exyz
  close(u)
  allocate(z_ifc(nlev + 1))
  open(newunit=u, file="z_ifc.bin", access="stream", form="unformatted", status="old")
  read(u) z_ifc
  close(u)
  allocate(vn(nlev, ne), w(nlev + 1, nc), rho(nlev, nc), exner(nlev, nc), theta(nlev, nc), exner_pr(nlev, nc))
  open(newunit=u, file="state.bin", access="stream", form="unformatted", status="old")
  read(u) vn, w, rho, exner, theta, exner_pr
  close(u)

  desc = icon_grid_desc_t(nc, ne, nv, 0, 6.371229d6, c_loc(c2v), c_loc(c2e), c_loc(e2c), c_loc(e2v), &
                          c_loc(v2e), c_loc(v2c), c_loc(cxyz), c_loc(vxyz), c_loc(exyz))
  rc = icon_grid_create(desc, grid)
  if (rc /= ICON_OK) stop 1
  call icon_dycore_params_default(params)
  params%dtime = 1800.0d0
  params%synchronous = 1
  params%autotune = 0
  rc = icon_dycore_create(grid, nlev, z_ifc, params, dycore)
  if (rc /= ICON_OK) then
    print *, icon_last_error_string()
    stop 2
  end if
  state = icon_state_t(c_loc(vn), c_loc(w), c_loc(rho), c_loc(exner), c_loc(theta), c_loc(exner_pr))
  do step = 1, 2
    rc = icon_dycore_step(dycore, state)
    if (rc /= ICON_OK) stop 3
  end do
  print *, "stepped; vn(1, 1) =", vn(1, 1)
  open(newunit=u, file="out.bin", access="stream", form="unformatted", status="replace")
  write(u) vn, w, rho, exner, theta, exner_pr
  close(u)
  rc = icon_dycore_destroy(dycore)
  rc = icon_grid_destroy(grid)
end program example_step
