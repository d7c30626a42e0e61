"""GB300-native volumetric PROPELLER reconstruction (sm_103a CUDA library + binding).

The compute lives in ``lib/libprop.so`` (built from ``csrc/`` by
:mod:`paper_2311_13177_gb300.build`); the modules here only marshal
arguments.  Importing the package does not load the library; the first call
does, and it raises if the library is missing.
"""
from .binding import (Plan, ReconParams, ProjParams, prop_plan_create, prop_plan_destroy, prop_plan_workspace_bytes,
                      prop_forward, prop_adjoint, prop_reconstruct, prop_reconstruct_host, prop_loss_grad,
                      prop_render, prop_psnr, prop_reconstruct_batch)
from .autograd import PropOp, prop_apply

__all__ = ["Plan", "ReconParams", "ProjParams", "prop_plan_create", "prop_plan_destroy", "prop_plan_workspace_bytes",
           "prop_forward", "prop_adjoint", "prop_reconstruct", "prop_reconstruct_host", "prop_loss_grad",
           "prop_render", "prop_psnr", "prop_reconstruct_batch", "PropOp", "prop_apply"]
