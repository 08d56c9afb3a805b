"""GB300-native Montgomery multiplication, NTT and polynomial multiplication.

The computation runs in hand-written sm_103a CUDA kernels behind the C ABI of
``include/mont.h`` (``libmontgomery.so``); this package is the thin Python
binding over that ABI, with the same names.  Build the library with
``paper_1609_00999_gb300.build.build()``.
"""
from ._binding import (MONT_ECUDA, MONT_EINVAL, MONT_ENOMEM, MONT_ERANGE, MONT_ETIMEOUT,  # noqa: F401
                       MONT_EUNSUPPORTED, MONT_OK, NTT_BITREV, MontCtx, MontError, NttPlan, from_mont,
                       lib, mont_fma, mont_mul, mont_setup, ntt_fwd, ntt_inv, ntt_plan_create, polymul,
                       polymul_many, strerror, to_mont)
from ._binding import mont_release_workspaces, polymul_many_ws, polymul_noalloc, polymul_workspace_bytes  # noqa: F401
from ._binding import polymul_many_fourier  # noqa: F401
from ._binding import (PolymulBatchConfig, PolymulBatchPlan, PolymulDesc,  # noqa: F401
                       polymul_batch, polymul_batch_check, polymul_batch_describe, polymul_batch_plan_create,
                       polymul_batch_workspace_bytes)
from ._binding import MontServer, MontServerStats, completion_dtype, request_dtype  # noqa: F401
from ._binding import barrett_mulmod, check_residues, fourier_redc_mul  # noqa: F401
from ._binding import PROBE_KINDS, int_probe  # noqa: F401
