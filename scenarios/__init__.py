"""Seeded synthetic workloads for the fixed-step cable-network engine.

This package only draws inputs: morphologies (segment length, diameter, axial
resistivity, specific capacitance), mechanism placement and parameters,
NetCon wiring, external event trains and stimuli.  It performs none of the
simulation arithmetic (no areas, couplings, currents or solves), so it can feed
both the CUDA engine and the CPU oracle without sharing any of their code.
"""
from .generator import (Scenario, MechTable, ring16, network, batched, adjoint_net, morph_types,
                        passive_cable, single_compartment, MECH_PARAMS)

__all__ = ["Scenario", "MechTable", "ring16", "network", "batched", "adjoint_net", "morph_types",
           "passive_cable", "single_compartment", "MECH_PARAMS"]
