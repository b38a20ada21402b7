"""Seeded synthetic SUR inputs shared by the oracle and the CUDA path."""
