"""GB300-native network density of states (KPM Chebyshev moments).

Python face of the CUDA library ``libnetdos.so`` (C ABI: include/netdos.h).
The functions carry the ABI's names; see ``_binding`` for their arguments.
"""
from ._binding import (  # noqa: F401
    DOS_EINVAL,
    DOS_ENOMEM,
    DOS_OK,
    DosError,
    Filter,
    Graph,
    density_with_spikes,
    dos_autotune,
    dos_batch_info,
    dos_build_csr,
    dos_build_csr_batched,
    dos_density,
    dos_device_status,
    dos_filter_export,
    dos_filter_info,
    dos_get_plan,
    dos_graph_export,
    dos_graph_info,
    dos_launch_count,
    dos_moments,
    dos_moments_batched,
    dos_moments_noalloc,
    dos_motif_filter,
    dos_profile_enable,
    dos_profile_read,
    dos_set_plan,
    dos_version,
    header_functions,
    ldos_moments,
    lib,
)
