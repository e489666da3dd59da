"""GB300-native SLM split search with particle swarm optimisation.

The computation lives in ``libslm.so`` (hand-written sm_103a CUDA behind the C
ABI declared in ``include/slm.h``); ``binding`` marshals arguments to it.
``workloads`` draws the synthetic inputs.
"""
__all__ = ["binding", "build", "workloads"]
