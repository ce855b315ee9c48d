"""Seeded synthetic inputs shared by the CPU oracle and the GPU library: networks,
contraction paths and slicing metadata. Holds no contraction arithmetic."""
from .network import Network, Path, relabel_compact
from . import circuits, kicked_ising, ising_pf, greedy, workloads

__all__ = ["Network", "Path", "relabel_compact", "circuits", "kicked_ising", "ising_pf",
           "greedy", "workloads"]
