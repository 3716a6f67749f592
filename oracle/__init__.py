"""FP64 CPU oracle (test infrastructure only; never imported by the library)."""

from . import seg_oracle  # noqa: F401
