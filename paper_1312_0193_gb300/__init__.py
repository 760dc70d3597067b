"""GB300 (sm_103a) implementation of the SGD hot path of NOMAD
(Yun et al., arXiv 1312.0193): a persistent CUDA kernel in which every warp
is a NOMAD worker and item vectors circulate as tokens between device-side
queues, behind the C ABI of include/nomad.h.  See ``nomad.Nomad``."""
from .nomad import (Nomad, NomadError, load_library, LIB_PATH,  # noqa: F401
                    nomad_schedule, nomad_info, nomad_schedule_default,
                    nomad_create, nomad_load_ratings, nomad_epoch, nomad_epoch_many,
                    nomad_check,
                    nomad_rmse, nomad_objective, nomad_get_factors,
                    nomad_set_factors, nomad_get_info, nomad_destroy)
