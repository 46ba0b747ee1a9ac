"""FP64 CPU oracle (test infrastructure only; see ``upols_oracle``)."""
from .upols_oracle import (  # noqa: F401
    UpolsOracle,
    afc_closed_loop,
    afc_closed_loop_reuse,
    mimo_fir,
    mimo_fir_sample,
    num_partitions,
    upols,
)
