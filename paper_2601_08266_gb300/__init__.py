"""GB300-native hot path of the immersed FSI method of arxiv 2601.08266.

The operators live in the CUDA library ``libfsi.so`` (C ABI: include/fsi.h);
this package only builds it (``build.build``), binds it (``_binding``) and
provides seeded synthetic inputs (``inputs``).
"""
from ._binding import (FSI_BATCH_GRAPH, FSI_BATCH_PER_INSTANCE, FSI_BATCH_PERSISTENT,  # noqa: F401
                       FSI_DF64, FSI_F32, FSI_F64, Batch, FsiError, Mesh, Mlp, StepState,
                       fsi_mesh_set_brick, fsi_mesh_autotune, fsi_residual_jacobian_apply,
                       fsi_mlp_adam, fsi_mlp_features, fsi_mlp_forward, fsi_mlp_loss_grad,
                       fsi_mlp_num_params, fsi_mlp_predict, fsi_mlp_guess,
                       fsi_advance_history,
                       fsi_block_diagonal, fsi_coupled_jacobian_apply, fsi_coupled_residual,
                       fsi_dlm_interp, fsi_dlm_spread, fsi_jacobian_apply, fsi_locate,
                       fsi_locate_noalloc, fsi_newton_step, fsi_residual, fsi_stage, lib,
                       library_path, PRECOND_BLOCK_JACOBI, PRECOND_SCHUR, fsi_interface_scaling,
                       fsi_mesh_set_coordinates,
                       TetMesh, MeshTet, fsi_tet_residual, fsi_tet_jacobian_apply, fsi_tet_locate,
                       fsi_tet_interp, fsi_tet_spread, fsi_wait_selftest,
                       Solid, fsi_solid_residual, fsi_solid_tangent_apply, fsi_solid_stage,
                       fsi_solid_advance, fsi_solid_positions,
                       fsi_pressure_levels, fsi_pressure_set_faces, fsi_pressure_apply, fsi_pressure_restrict,
                       fsi_pressure_prolong_add, fsi_pressure_smooth, fsi_pressure_vcycle,
                       fsi_pressure_level_sizes, fsi_pressure_set_eliminated,
                       fsi_pressure_use_amg)
