"""GB300-native GDI annealer for balanced min-cut bisection (Cook, Jin, Tan, arXiv:1908.00210).

The compute path is libgdi.so (hand-written sm_103a CUDA behind the C ABI of include/gdi.h);
this package only marshals arguments to it.
"""
from ._binding import (  # noqa: F401
    EXPORTS, GDI_FLAG_CONTINUE, GDI_FLAG_NO_REPAIR, GDI_FLAG_RACY, GDI_FLAG_STANDARD, GDI_FLAG_TRACE, GDI_MEM_DEVICE, GDI_MEM_HOST,
    GDI_METROPOLIS, GDI_PAPER_PF, GDI_PATH_AUTO, GDI_PATH_CTA, GDI_PATH_GRID, LIB_PATH, Annealer,
    GdiError, RankSpace, Schedule, build_table, load, rank_space,
)
from .build import build  # noqa: F401
