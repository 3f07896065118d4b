"""libcht: a GB300-native concurrent hash table (folklore linear probing,
Maier, Sanders & Dementiev, arXiv 1601.04017) behind a C ABI.

The compute path is hand-written CUDA for sm_103a in ``csrc/``, built into
``libcht.so`` in this directory; this package only marshals arguments.
"""
from ._build import build
from .cht import (OP_ERASE, OP_FIND, OP_INSERT, OP_IOU_ADD, OP_IOU_OVERWRITE, OP_UPDATE_ADD, OP_UPDATE_OVERWRITE,
                  PLAN_TIMEOUT, Plan, Server, ADD, CHT_ERR_CUDA, CHT_ERR_INVALID_ARG, CHT_ERR_OOM, CHT_ERR_RESERVED_KEY,
                  CHT_ERR_TABLE_FULL, CHT_ERR_TIMEOUT, CHT_OK, CODE_FULL, CODE_NO, CODE_RESERVED,
                  CODE_YES, OVERWRITE, STATUS_FULL, STATUS_RESERVED, ChtError, Table, launch_count,
                  library_path, load_library, memory_in_use, set_memory_limit, version)

__all__ = [
    "ADD", "OVERWRITE", "Table", "Plan", "Server", "OP_FIND", "OP_INSERT", "OP_IOU_ADD", "OP_IOU_OVERWRITE", "OP_ERASE", "OP_UPDATE_ADD", "OP_UPDATE_OVERWRITE",
    "PLAN_TIMEOUT", "ChtError", "build", "load_library", "library_path", "launch_count",
    "memory_in_use", "set_memory_limit", "version", "CHT_OK", "CHT_ERR_INVALID_ARG", "CHT_ERR_OOM",
    "CHT_ERR_CUDA", "CHT_ERR_TABLE_FULL", "CHT_ERR_RESERVED_KEY", "CHT_ERR_TIMEOUT", "CODE_NO",
    "CODE_YES", "CODE_FULL", "CODE_RESERVED", "STATUS_FULL", "STATUS_RESERVED",
]
