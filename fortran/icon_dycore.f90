! Fortran interface to libicondycore (include/icon_dycore.h): the C-ABI a
! host model such as ICON calls (Sec. 4.3: arrays by reference, scalars by
! value, logical flags as 32-bit integers).  Every routine is the C function
! of the same name; see the header for argument meaning, layout, ownership
! and error codes.  Level-contiguous library arrays are the Fortran arrays
! X(nlev_x, n_points); nproma-blocked ICON arrays X(nproma, nlev_x, nblks) go
! through icon_state_from_blocked / icon_state_to_blocked /
! icon_dycore_step_blocked.
module icon_dycore
  use, intrinsic :: iso_c_binding
  implicit none
  private

  integer(c_int), parameter, public :: ICON_OK = 0, ICON_ERR_ARG = -1, ICON_ERR_CUDA = -2, &
       ICON_ERR_GRID = -3, ICON_ERR_NUMERIC = -4, ICON_ERR_UNSUPPORTED = -5
  integer(c_int32_t), parameter, public :: ICON_PREC_FP64 = 0, ICON_PREC_MIXED = 1, ICON_PREC_MIXED_F64COL = 2

  type, bind(c), public :: icon_grid_desc_t
    integer(c_int32_t) :: n_cells, n_edges, n_verts, index_base
    real(c_double) :: sphere_radius
    type(c_ptr) :: c2v, c2e, e2c, e2v, v2e, v2c, cell_xyz, vert_xyz, edge_xyz
  end type

  type, bind(c), public :: icon_dycore_params_t
    real(c_double) :: dtime
    integer(c_int32_t) :: ndyn_substeps
    real(c_double) :: grav, rd, cpd, p00, omega
    real(c_double) :: vwind_impl_wgt, wgt_nnow_vel, wgt_nnew_vel, wgt_nnow_rth, wgt_nnew_rth
    real(c_double) :: exner_exfac, divdamp_fac, divflux_fac, rayleigh_coeff, damp_height
    real(c_double) :: hdiff_smag_fac, hdiff_k4, hdiff_w_k4
    integer(c_int32_t) :: hdiff_temp
    real(c_double) :: ref_T0
    integer(c_int32_t) :: precision, use_graph, autotune, synchronous
    type(c_ptr) :: stream
    integer(c_int32_t) :: column_chunk
    integer(c_int32_t) :: steep_hpg
    real(c_double) :: hdiff_tenh_fac, hdiff_tenh_thresh
    integer(c_int32_t) :: hdiff_tenh_levels
    integer(c_int32_t) :: fused_advection
  end type

  type, bind(c), public :: icon_state_t
    type(c_ptr) :: vn, w, rho, exner, theta_v, exner_pr
  end type

  public :: icon_grid_create, icon_grid_destroy, icon_dycore_params_default, icon_dycore_create, &
       icon_dycore_create_terrain, icon_dycore_reference_columns, icon_dycore_destroy, icon_dycore_step, icon_nh_solve, icon_nh_diff, icon_dycore_diagnostics, &
       icon_state_from_blocked, icon_state_to_blocked, icon_dycore_step_blocked, icon_last_error_string, &
       icon_dycore_save, icon_dycore_load

  interface
    integer(c_int) function icon_grid_create(desc, grid) bind(c, name="icon_grid_create")
      import :: c_int, c_ptr, icon_grid_desc_t
      type(icon_grid_desc_t), intent(in) :: desc
      type(c_ptr), intent(out) :: grid
    end function
    integer(c_int) function icon_grid_destroy(grid) bind(c, name="icon_grid_destroy")
      import :: c_int, c_ptr
      type(c_ptr), value :: grid
    end function
    subroutine icon_dycore_params_default(params) bind(c, name="icon_dycore_params_default")
      import :: icon_dycore_params_t
      type(icon_dycore_params_t), intent(out) :: params
    end subroutine
    integer(c_int) function icon_dycore_create(grid, nlev, z_ifc, params, dycore) bind(c, name="icon_dycore_create")
      import :: c_int, c_int32_t, c_double, c_ptr, icon_dycore_params_t
      type(c_ptr), value :: grid
      integer(c_int32_t), value :: nlev
      real(c_double), intent(in) :: z_ifc(*)
      type(icon_dycore_params_t), intent(in) :: params
      type(c_ptr), intent(out) :: dycore
    end function
    ! terrain-following heights per column: z_ifc(nlev+1, n_cells)
    integer(c_int) function icon_dycore_create_terrain(grid, nlev, z_ifc, params, dycore) &
        bind(c, name="icon_dycore_create_terrain")
      import :: c_int, c_int32_t, c_double, c_ptr, icon_dycore_params_t
      type(c_ptr), value :: grid
      integer(c_int32_t), value :: nlev
      real(c_double), intent(in) :: z_ifc(*)
      type(icon_dycore_params_t), intent(in) :: params
      type(c_ptr), intent(out) :: dycore
    end function
    ! reference theta_v and exner per column: (nlev, n_cells) each
    integer(c_int) function icon_dycore_reference_columns(dycore, theta_ref, exner_ref) &
        bind(c, name="icon_dycore_reference_columns")
      import :: c_int, c_double, c_ptr
      type(c_ptr), value :: dycore
      real(c_double), intent(out) :: theta_ref(*), exner_ref(*)
    end function
    integer(c_int) function icon_dycore_destroy(dycore) bind(c, name="icon_dycore_destroy")
      import :: c_int, c_ptr
      type(c_ptr), value :: dycore
    end function
    integer(c_int) function icon_dycore_step(dycore, state) bind(c, name="icon_dycore_step")
      import :: c_int, c_ptr, icon_state_t
      type(c_ptr), value :: dycore
      type(icon_state_t), intent(in) :: state
    end function
    ! checkpoint / restart; path is a NUL-terminated character array (trim(name)//c_null_char)
    integer(c_int) function icon_dycore_save(dycore, state, path) bind(c, name="icon_dycore_save")
      import :: c_int, c_ptr, c_char, icon_state_t
      type(c_ptr), value :: dycore
      type(icon_state_t), intent(in) :: state
      character(kind=c_char), dimension(*), intent(in) :: path
    end function
    integer(c_int) function icon_dycore_load(dycore, state, path) bind(c, name="icon_dycore_load")
      import :: c_int, c_ptr, c_char, icon_state_t
      type(c_ptr), value :: dycore
      type(icon_state_t), intent(in) :: state
      character(kind=c_char), dimension(*), intent(in) :: path
    end function
    integer(c_int) function icon_nh_solve(dycore, state) bind(c, name="icon_nh_solve")
      import :: c_int, c_ptr, icon_state_t
      type(c_ptr), value :: dycore
      type(icon_state_t), intent(in) :: state
    end function
    integer(c_int) function icon_nh_diff(dycore, state) bind(c, name="icon_nh_diff")
      import :: c_int, c_ptr, icon_state_t
      type(c_ptr), value :: dycore
      type(icon_state_t), intent(in) :: state
    end function
    integer(c_int) function icon_dycore_diagnostics(dycore, state, ps, t850, mass) &
         bind(c, name="icon_dycore_diagnostics")
      import :: c_int, c_ptr, c_double, icon_state_t
      type(c_ptr), value :: dycore
      type(icon_state_t), intent(in) :: state
      type(c_ptr), value :: ps, t850
      real(c_double), intent(out) :: mass
    end function
    integer(c_int) function icon_state_from_blocked(dycore, nproma, blocked, state) &
         bind(c, name="icon_state_from_blocked")
      import :: c_int, c_int32_t, c_ptr, icon_state_t
      type(c_ptr), value :: dycore
      integer(c_int32_t), value :: nproma
      type(icon_state_t), intent(in) :: blocked, state
    end function
    integer(c_int) function icon_state_to_blocked(dycore, nproma, state, blocked) &
         bind(c, name="icon_state_to_blocked")
      import :: c_int, c_int32_t, c_ptr, icon_state_t
      type(c_ptr), value :: dycore
      integer(c_int32_t), value :: nproma
      type(icon_state_t), intent(in) :: state, blocked
    end function
    integer(c_int) function icon_dycore_step_blocked(dycore, nproma, blocked) bind(c, name="icon_dycore_step_blocked")
      import :: c_int, c_int32_t, c_ptr, icon_state_t
      type(c_ptr), value :: dycore
      integer(c_int32_t), value :: nproma
      type(icon_state_t), intent(in) :: blocked
    end function
    type(c_ptr) function icon_last_error_c() bind(c, name="icon_last_error")
      import :: c_ptr
    end function
  end interface

contains

  ! The message of the last failing call on this thread as a Fortran string.
  function icon_last_error_string() result(msg)
    character(len=:), allocatable :: msg
    character(kind=c_char), pointer :: chars(:)
    integer :: n
    type(c_ptr) :: p
    p = icon_last_error_c()
    n = 0
    if (c_associated(p)) then
      call c_f_pointer(p, chars, [4096])
      do while (n < 4096)
        if (chars(n + 1) == c_null_char) exit
        n = n + 1
      end do
    end if
    allocate(character(len=n) :: msg)
    if (n > 0) msg = transfer(chars(1:n), msg)
  end function

end module icon_dycore
